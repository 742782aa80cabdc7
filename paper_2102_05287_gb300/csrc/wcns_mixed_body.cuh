// Mixed-precision sweep body: the same RHS as sweep_body (wcns_sweep.cuh)
// arranged for GB300's 61:1 FP32:FP64 throughput.
//
// FP64 is kept where the method needs it: the node pressure (p + p_inf
// cancellation), the stored midpoint fluxes and the cell update (so the
// conserved components still telescope to FP64 round-off), the SSPRK3
// combine, and the limiters' theta solves.  Everything else runs in FP32 in
// deviation form about node i:
//   * node prep splits every primitive value and flux into an FP32 pair
//     (hi, lo) with hi + lo = value (hi truncated to 24 bits, lo the exact
//     remainder rounded), using integer bit operations, so a deviation
//     (hi_j - hi_i) + (lo_j - lo_i) is accurate to FP32 relative precision
//     of the deviation itself;
//   * projection, WCNS-IS, back-projection, both HLLC fluxes and the HCS
//     reconstruction work on deviations (hllc_dev, hcs);
//   * the limiters first try to certify in FP32, with a rigorous margin,
//     that every quantity the paper tests (partial densities, volume
//     fractions, rho ctilde^2) of every interpolated state and half state is
//     at least its tolerance; then every theta is 1 exactly as in FP64 and
//     nothing else is needed.  Otherwise the FP64 limiter code runs on FP64
//     states rebuilt from the same deviations.
#pragma once
#include <type_traits>

#include "wcns_sweep.cuh"

namespace wcns {

// Resident blocks per SM the register allocation targets: 4 in 2D (256
// threads, 64 registers), 3 in 3D (192 threads, 96 registers) and 8 for the
// 3D 128-thread x tiles (64 registers), 2 in 1D (128 threads).  Shared
// memory holds three 2D tiles and six 3D x tiles per SM.  In 2D the 64-
// register build keeps the same three blocks and still runs 3 % faster per
// sweep than 80 registers, despite its spills; the 3D x tiles at 64
// registers reach the six blocks that shared memory allows (five at 96
// registers), 10 % faster.  48 registers (2D) and 51 (3D x) run slower
// again.
#ifndef MIXED_MIN_BLOCKS
#define MIXED_MIN_BLOCKS 2
#endif
#ifndef MIXED_MIN_BLOCKS_2D
#define MIXED_MIN_BLOCKS_2D 4
#endif
#ifndef MIXED_MIN_BLOCKS_3D
#define MIXED_MIN_BLOCKS_3D 3
#endif

// Tile shapes (lines x midpoints): x sweeps 2 x 123 with 256 threads,
// 1D 1 x 123 with 128 threads and 2D y sweeps 4 x 59 (x-columns x
// midpoints) with 256 threads, so that the node stage (midpoints + 5 nodes
// a line) is exactly one node per thread.  4 x 59 has 8 % halo nodes
// against 19 % for 8 x 27 and measured 3 % faster per y sweep (2 x 123:
// 3 % slower; 8 x 32, whose 296 nodes take two rounds: 1.6 % slower per
// step than 8 x 27).
#ifndef MIXED_TL_X
#define MIXED_TL_X 2
#endif
#ifndef MIXED_TM_X
#define MIXED_TM_X (256 / MIXED_TL_X - 5)
#endif
#ifndef MIXED_TM_1D
#define MIXED_TM_1D 123
#endif
#ifndef MIXED_TL_Y
#define MIXED_TL_Y 4
#endif
#ifndef MIXED_TM_Y
#define MIXED_TM_Y (256 / MIXED_TL_Y - 5)
#endif
template <int NDIM, int DIR>
using TileMixed2 = TileT<(DIR == 0) ? (NDIM == 1 ? 1 : MIXED_TL_X) : MIXED_TL_Y,
                         (DIR == 0) ? (NDIM == 1 ? MIXED_TM_1D : MIXED_TM_X) : MIXED_TM_Y,
                         (DIR == 0) ? (NDIM == 1 ? 128 : 256) : 256>;
// 3D tiles (seven fields a node, 232 bytes of shared memory per node) have
// their own shape: y/z tiles 8 x 24 (192 midpoints) with 192 threads, 67 KB,
// three blocks per SM (measured on the 3D bubble collapse: 10 % faster than
// 256-thread tiles at two blocks per SM); x tiles 2 x 59 (128 nodes) with
// 128 threads, six blocks per SM (4 % faster there than 3 x 59 or 2 x 91
// at 192 threads; 2 x 59 y/z tiles measured 30 % slower).
#ifndef MIXED3_THREADS
#define MIXED3_THREADS 192
#endif
#ifndef MIXED3_TL_Y
#define MIXED3_TL_Y 8
#endif
#ifndef MIXED3_TM_Y
#define MIXED3_TM_Y (MIXED3_THREADS / MIXED3_TL_Y)
#endif
template <int NDIM, int DIR>
using TileMixed = typename std::conditional<
    NDIM == 3,
    typename std::conditional<DIR == 0, TileT<2, 59, 128>, TileT<MIXED3_TL_Y, MIXED3_TM_Y, MIXED3_THREADS>>::type,
    TileMixed2<NDIM, DIR>>::type;

// value = hi + lo: hi keeps the leading 24 bits of the double (truncated),
// lo is the exact remainder rounded to FP32.  Integer operations only, so
// the FP64 pipe is not involved.  Magnitudes below FP32's normal range
// (2^-126, never met by admissible states apart from exact zeros) give
// hi = lo = 0 with the sign kept; magnitudes above it give hi = +-inf (NaN
// stays NaN), lo = 0.
__device__ __forceinline__ void split_hilo(double v, float &hi, float &lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FFull);
  const int e32 = e - 1023 + 127;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (e32 <= 0 || e32 >= 255) {
    const unsigned int nan = (e == 0x7FF && m) ? 0x400000u : 0u;
    hi = __uint_as_float(e32 <= 0 ? sign : (sign | 0x7F800000u | nan));
    lo = 0.0f;
    return;
  }
  hi = __uint_as_float(sign | ((unsigned int)e32 << 23) | (unsigned int)(m >> 29));
  const unsigned int low = (unsigned int)(m & 0x1FFFFFFFull);
  const int es = e - 1075 + 127;  // exponent of the last mantissa bit, biased for FP32
  const float scale = es > 0 ? __uint_as_float((unsigned int)es << 23) : 0.0f;
  lo = __uint_as_float(__float_as_uint((float)low * scale) | sign);
}

// FP32 -> FP64 on the integer pipe (the FP64 pipe is the scarce one):
// exact for normal numbers, zeros, infinities and NaNs; FP32 subnormals
// (below 1.2e-38) become zeros of the same sign.
__device__ __forceinline__ double f2d(float x) {
  const unsigned int b = __float_as_uint(x);
  const unsigned int e = (b >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  if (e == 0u) return __longlong_as_double((long long)sign);
  const unsigned long long e64 = e == 0xFFu ? 0x7FFull : (unsigned long long)(e + 896u);
  const unsigned long long m = (unsigned long long)(b & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(sign | (e64 << 52) | m));
}

// 1/y for the mixed path's FP64 node work: Newton-Raphson refinement
// r <- r + r (1 - y r) of an FP32 seed.  The seed, the correctly rounded
// FP32 reciprocal of y's leading 24 bits, is within ~2^-22 of 1/y; one step
// squares that to ~2^-44, far below the FP32 precision the rest of the
// mixed path carries.  y must be finite, nonzero and within FP32's normal
// range (densities and Gamma of admissible states are).
__device__ __forceinline__ double recip_nr(double y) {
  float hi, lo;
  split_hilo(y, hi, lo);
  const double r = f2d(__frcp_rn(hi));
  return fma(r, fma(-y, r, 1.0), r);
}

// Shared-memory layout of a mixed tile.
template <int NDIM, class T>
struct SmemMixed {
  static constexpr int NF = NDIM + 4;
  // FP64: W, G per node; FP32: V hi/lo, G hi/lo per node, c, node flags
  static constexpr size_t NODE_BYTES = 8 * 2 * NF + 4 * 4 * NF + 4 + 4;
  static constexpr size_t MID_BYTES = 8 * (NF + 1);
  // + per-block scalars: dt, lambda, b dt, b dt / dx, 2 lambda (FP32)
  // + the list of midpoints deferred to the FP64 fallback pass and its length
  static constexpr size_t BYTES = NODE_BYTES * T::NN + MID_BYTES * T::NM + 5 * 8 + 4 * T::NM + 16;
  double *W, *G, *F, *am, *ap, *scal;
  float *Vh, *Vl, *Gh, *Gl, *c;
  unsigned int *ok, *nslow;
  int *slow;
  __device__ SmemMixed(double *base) {
    W = base;
    G = W + NF * T::NN;
    F = G + NF * T::NN;
    am = F + (NF - 1) * T::NM;
    ap = am + T::NM;
    Vh = (float *)(ap + T::NM);
    Vl = Vh + NF * T::NN;
    Gh = Vl + NF * T::NN;
    Gl = Gh + NF * T::NN;
    c = Gl + NF * T::NN;
    ok = (unsigned int *)(c + T::NN);
    scal = (double *)(ok + T::NN);  // c and ok together take 8 NN bytes: 8-byte aligned
    slow = (int *)(scal + 5);
    nslow = (unsigned int *)(slow + T::NM);
  }
};

// Certification margin: FP32 evaluation of a short expression over terms of
// total magnitude `mag` is within 2^-20 * mag of the exact value (a handful
// of roundings at 2^-24 each).
__device__ __forceinline__ float margin(float mag) { return 9.5367431640625e-07f * mag; }

// FP32 check that rho ctilde^2 = E - |m|^2/(2 rho) - pbar(alpha1) (Sec. 2)
// of a conservative state is >= eps, given an FP32 state x whose every
// component lies within margin(mag[f]) of the exact one.  Each error is
// propagated: rho, the kinetic energy (through m and rho), pbar (through
// alpha1, with |d pbar / d alpha1| = q1 (r2 + 1)/(Gamma + 1)^2 <= q1 (r2 + 1)),
// and the FP32 evaluation itself.  Returns true only if certain.
template <int NDIM>
__device__ __forceinline__ bool rct2_certified(const EosConst &e, const float *x, const float *mag, float eps) {
  constexpr int E = 2 + NDIM, A = 3 + NDIM;
  const float rho = x[0] + x[1];
  const float drho = margin(mag[0] + mag[1] + fabsf(rho));
  const float rlo = rho - drho;
  if (!(rlo > 0.0f)) return false;
  float m2 = 0.0f, dm2 = 0.0f;
#pragma unroll
  for (int j = 0; j < NDIM; ++j) {
    const float mj = x[2 + j], dm = margin(mag[2 + j]);
    m2 += mj * mj;
    dm2 += (2.0f * fabsf(mj) + dm) * dm;
  }
  const float ke = 0.5f * __fdividef(m2, rho);
  const float dke = 0.5f * __fdividef(dm2, rlo) + __fdividef(ke * drho, rlo) + margin(ke);
  const float al = x[A];
  const float Gam = e.r2f + e.drf * al;
  const float pb = __fdividef(e.q1f * al, Gam + 1.0f);
  const float dpb = e.q1f * (e.r2f + 1.0f) * margin(mag[A]) + margin(pb);
  const float v = x[E] - ke - pb;
  return v - (margin(mag[E]) + dke + dpb + margin(fabsf(x[E]) + ke + pb)) >= eps;
}

// FP64 velocity, pressure and sound speed of a node from its conservative
// state (Sec. 2), with the FP64 sweep's formulas.
template <int NDIM>
__device__ __forceinline__ void node_thermo64(const EosConst &eos, const double *w, double *v, double &p,
                                              double &c) {
  constexpr int E = 2 + NDIM, A = 3 + NDIM;
  const double rho = w[0] + w[1];
  const double ir = 1.0 / rho;
  double m2 = 0.0;
#pragma unroll
  for (int j = 0; j < NDIM; ++j) {
    v[j] = w[2 + j] * ir;
    m2 = fma(w[2 + j], v[j], m2);
  }
  const double rhoe = w[E] - 0.5 * m2;
  const double Gam = mixGamma(eos, w[A]);
  const double Pi = mixPi(eos, w[A]);
  const double x = 1.0 / (Gam * (Gam + 1.0));
  const double iG = (Gam + 1.0) * x;
  p = (rhoe - Pi) * iG;
  c = sqrt(((Gam + 1.0) * rhoe - Pi) * (iG * iG) * ir);
}

// Small vectors passed by value to the out-of-line FP64 fallbacks below.
template <int N>
struct FVec {
  float v[N];
};
template <int NF>
struct LimitedState {
  float d[NF];  // deviation of the limited state from node i
  float c;      // its sound speed
  int flags;    // interp_limit flags (0: unchanged, d and c not set)
};

// FP64 interpolation limiter of the mixed path (Sec. 5.1, Algorithms 1-3),
// taken where the FP32 certification fails: node k's FP64 state Wn
// (shared memory, stride nn), the interpolated state rebuilt in FP64 from
// node i's hi/lo parts plus the deviation d, V -> W, then the limiter; a
// limited state comes back as a deviation from node i and its sound speed.
// Out of line so that its FP64 registers do not shape the FP32 fast path's
// register allocation.
template <int NDIM>
__device__ __noinline__ LimitedState<NDIM + 4> mixed_interp_fallback(const EosConst eos, const LimTol tol,
                                                                      const double *Wsm, int nn, int nk,
                                                                      const FVec<NDIM + 4> hi_i,
                                                                      const FVec<NDIM + 4> lo_i,
                                                                      const FVec<NDIM + 4> d) {
  constexpr int NF = NDIM + 4, E = 2 + NDIM, A = 3 + NDIM;
  LimitedState<NF> out;
  double Wn[NF], Wt[NF], V[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    Wn[f] = Wsm[f * nn + nk];
    V[f] = ((double)hi_i.v[f] + (double)lo_i.v[f]) + (double)d.v[f];
  }
  const double rho = V[0] + V[1];
  double k2s = 0.0;
#pragma unroll
  for (int k = 0; k < NDIM; ++k) {
    Wt[2 + k] = rho * V[2 + k];
    k2s = fma(V[2 + k], V[2 + k], k2s);
  }
  Wt[0] = V[0];
  Wt[1] = V[1];
  Wt[E] = fma(V[E], mixGamma(eos, V[A]), mixPi(eos, V[A])) + 0.5 * rho * k2s;
  Wt[A] = V[A];
  out.flags = interp_limit<NDIM>(eos, tol, Wn, Wt);
  if (out.flags) {
    const double r = Wt[0] + Wt[1];
    const double ir = 1.0 / r;
    double mm = 0.0, vv[NDIM];
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
      vv[k] = Wt[2 + k] * ir;
      mm = fma(Wt[2 + k], vv[k], mm);
    }
    const double pn = (Wt[E] - 0.5 * mm - mixPi(eos, Wt[A])) / mixGamma(eos, Wt[A]);
    out.d[0] = (float)(Wt[0] - ((double)hi_i.v[0] + (double)lo_i.v[0]));
    out.d[1] = (float)(Wt[1] - ((double)hi_i.v[1] + (double)lo_i.v[1]));
#pragma unroll
    for (int k = 0; k < NDIM; ++k)
      out.d[2 + k] = (float)(vv[k] - ((double)hi_i.v[2 + k] + (double)lo_i.v[2 + k]));
    out.d[E] = (float)(pn - ((double)hi_i.v[E] + (double)lo_i.v[E]));
    out.d[A] = (float)(Wt[A] - ((double)hi_i.v[A] + (double)lo_i.v[A]));
    // sound speed of the limited state
    const double Gm_ = mixGamma(eos, Wt[A]);
    const double pb = mixPi(eos, Wt[A]) / (Gm_ + 1.0);
    out.c = (float)sqrt((1.0 + 1.0 / Gm_) * (pn + pb) * ir);
  }
  return out;
}

// FP64 flux limiter of the mixed path (Sec. 5.2, Algorithms 4-6), taken
// where the FP32 certification fails: on FP64 node states and the FP64
// first-order HLLC flux (its positivity is what the limiter falls back on,
// so it is not taken from the FP32 deviations).  The high-order split
// fluxes are rebuilt from node i's FP64 flux plus the FP32 deviations dGh;
// the limited G^-, G^+ are written to the midpoint's shared-memory slot
// (F: shared components, am / ap: alpha1 components).  Returns the
// flux_limit flags (a non-finite high-order flux takes the hard switch).
// Out of line for the same reason as mixed_interp_fallback.
template <int NDIM, int DIR>
__device__ __noinline__ int mixed_flux_fallback(const EosConst eos, const LimTol tol, const double *Wsm,
                                                const double *Gsm, int nn, int ni, int ni1, double *Fsm,
                                                double *am, double *ap, int nm, int ms, double ui64, float duh,
                                                const FVec<NDIM + 4> dGh, double lam) {
  constexpr int NF = NDIM + 4, A = 3 + NDIM;
  double Wi[NF], Wi1[NF], Fi[NF], Fi1[NF], GH[NF], uH, Gm[NF], Gp[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    Wi[f] = Wsm[f * nn + ni];
    Wi1[f] = Wsm[f * nn + ni1];
    Fi[f] = Gsm[f * nn + ni];
    Fi1[f] = Gsm[f * nn + ni1];
  }
#pragma unroll
  for (int f = 0; f < NF - 1; ++f) Gm[f] = Gp[f] = Fi[f] + f2d(dGh.v[f]);
  Fi[A] = Fi1[A] = 0.0;
  {
    double vi[NDIM], vi1[NDIM], pi_, pi1, ci_, ci1_;
    node_thermo64<NDIM>(eos, Wi, vi, pi_, ci_);
    node_thermo64<NDIM>(eos, Wi1, vi1, pi1, ci1_);
    hllc<NDIM, DIR, double>(Wi, vi, pi_, Wi[0] + Wi[1], ci_, Wi1, vi1, pi1, Wi1[0] + Wi1[1], ci1_, GH, uH);
  }
  double GHm[NF], GHp[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) GHm[f] = GHp[f] = GH[f];
  GHm[A] = GH[A] - Wi[A] * uH;
  GHp[A] = GH[A] - Wi1[A] * uH;
  const double uh64 = ui64 + (double)duh;
  Gm[A] = Gsm[A * nn + ni] + (double)dGh.v[A] - Wi[A] * uh64;
  Gp[A] = Gsm[A * nn + ni] + (double)dGh.v[A] - Wi1[A] * uh64;
  bool finite = true;
#pragma unroll
  for (int f = 0; f < NF; ++f) finite = finite && isfinite(Gm[f]) && isfinite(Gp[f]);
  int fl;
  if (finite) {
    fl = flux_limit<NDIM>(eos, tol, Wi, Wi1, Fi, Fi1, GHm, GHp, lam, Gm, Gp);
  } else {
    // a non-finite high-order flux: the hard switch of Sec. 5.2
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      Gm[f] = GHm[f];
      Gp[f] = GHp[f];
    }
    fl = 2;
  }
#pragma unroll
  for (int f = 0; f < NF - 1; ++f) Fsm[f * nm + ms] = Gm[f];
  am[ms] = Gm[A];
  ap[ms] = Gp[A];
  return fl;
}

// DEFER: midpoints whose FP32 certification fails are collected and
// computed in a second pass with the FP64 fallbacks (the grid sweeps);
// otherwise every midpoint runs the full code in one pass (the batched 1D
// kernels, whose persistent 64-thread tiles were measured faster that way).
template <int NDIM, int DIR, class T, bool DEFER = true, class Geo>
__device__ __forceinline__ void sweep_body_mixed(const SweepArgs &a, const Geo &geo, double *smem_raw) {
  using R = float;
  using S = SmemMixed<NDIM, T>;
  constexpr int NF = NDIM + 4, E = 2 + NDIM, A = 3 + NDIM;
  auto nslot = [](int l, int s) { return DIR == 0 ? l * T::NS + s : s * T::TL + l; };
  auto mslot = [](int l, int m) { return DIR == 0 ? l * T::TM + m : m * T::TL + l; };
  S sm(smem_raw);
  const int tid = threadIdx.x;
  const int tile0 = geo.tile0;
  const long long N = a.ncell;
  const EosConst eos = a.eos;
  const LimTol tol = a.tol;
  // the first sweep of an RHS (see mixed_first_dir)
  constexpr int FIRST = mixed_first_dir(NDIM);
  // Tolerances rounded up into FP32, so "x >= epsf" implies "x >= eps".
  const float epsf_ar = tol.cert_ar, epsf_a = tol.cert_a, epsf_rc = tol.cert_rc;

  // ---- 1+2: stage nodes, FP64 node work, hi/lo split -----------------------
  for (int q = tid; q < T::NN; q += T::THREADS) {
    const int l = DIR == 0 ? q / T::NS : q % T::TL;
    const int s = DIR == 0 ? q % T::NS : q / T::TL;
    const Line ln = geo.line(l);
    const int n = ln.n;
    const int pos = tile0 - 3 + s;
    double w[NF];
    bool dirichlet = false, flip = false;
    int src = pos;
    long long idx = 0;  // cell of a non-Dirichlet node
    if (pos < -3 || pos > n + 2) {
      src = min(max(pos, 0), n - 1);
    } else if (pos < 0 || pos >= n) {
      const int kind = pos < 0 ? a.bc_lo : a.bc_hi;
      if (kind == BC_TRANS) {
        src = pos < 0 ? 0 : n - 1;
      } else if (kind == BC_PERIODIC) {
        src = ((pos % n) + n) % n;
      } else if (kind == BC_SYMMETRY) {
        src = pos < 0 ? -1 - pos : 2 * n - 1 - pos;
        flip = true;
      } else {
        dirichlet = true;
      }
    }
    if (dirichlet) {
      const double *face = pos < 0 ? a.dir_face_lo : a.dir_face_hi;
      if (face) {
#pragma unroll
        for (int f = 0; f < NF; ++f) w[f] = __ldg(face + (long long)f * a.face_n + ln.face);
      } else if (pos < 0) {  // two direct loops: a selected pointer into the
#pragma unroll                     // parameter arrays would copy them to local memory
        for (int f = 0; f < NF; ++f) w[f] = a.dir_lo[f];
      } else {
#pragma unroll
        for (int f = 0; f < NF; ++f) w[f] = a.dir_hi[f];
      }
    } else {
      idx = ln.base + (long long)src * ln.stride;
#pragma unroll
      for (int f = 0; f < NF; ++f) w[f] = __ldg(a.W_in + (long long)f * N + idx);
      if (flip) w[2 + DIR] = -w[2 + DIR];
    }
    // Sec. 2 in FP64: p from rho e (the p + p_inf cancellation).  The later
    // sweeps of the same RHS load p and 1/rho of the node's cell from the
    // node cache (a symmetry ghost's mirrored momentum changes neither).
    bool cached = false;
    if constexpr (DIR != FIRST) cached = a.node_read && !dirichlet;
    double p, ir, v[NDIM];
    double adm_rct = 0.0;  // first sweep: (Gamma + 1) rho ctilde^2 and the other admissibility tests
    bool adm_ok = true;
    if (cached) {
      p = a.node_p[idx];
      ir = a.node_ir[idx];
#pragma unroll
      for (int j = 0; j < NDIM; ++j) v[j] = w[2 + j] * ir;
    } else {
      const double rho = w[0] + w[1];
      ir = recip_nr(rho);
      double m2 = 0.0;
#pragma unroll
      for (int j = 0; j < NDIM; ++j) {
        v[j] = w[2 + j] * ir;
        m2 = fma(w[2 + j], v[j], m2);
      }
      const double rhoe = w[E] - 0.5 * m2;
      const double Gam = mixGamma(eos, w[A]);
      const double Pi = mixPi(eos, w[A]);
      p = (rhoe - Pi) * recip_nr(Gam);
      adm_rct = rhoe * (Gam + 1.0) - Pi;  // (Gamma + 1) rho ctilde^2
      adm_ok = nonneg64(w[0]) && nonneg64(w[1]) && nonneg64(w[A]) &&
               __double_as_longlong(w[A]) <= 0x3FF0000000000000ll && finite64(rhoe) && finite64(p);
    }
    const double un = v[DIR];
    double g[NF];
    g[0] = w[0] * un;
    g[1] = w[1] * un;
#pragma unroll
    for (int j = 0; j < NDIM; ++j) g[2 + j] = w[2 + j] * un + (j == DIR ? p : 0.0);
    g[E] = (w[E] + p) * un;
    g[A] = w[A] * un;
    const int slot = nslot(l, s);
    float vh[NF], vl[NF];
    split_hilo(w[0], vh[0], vl[0]);
    split_hilo(w[1], vh[1], vl[1]);
#pragma unroll
    for (int j = 0; j < NDIM; ++j) split_hilo(v[j], vh[2 + j], vl[2 + j]);
    split_hilo(p, vh[E], vl[E]);
    split_hilo(w[A], vh[A], vl[A]);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      sm.W[f * T::NN + slot] = w[f];
      sm.G[f * T::NN + slot] = g[f];
      sm.Vh[f * T::NN + slot] = vh[f];
      sm.Vl[f * T::NN + slot] = vl[f];
      float gh, gl;
      split_hilo(g[f], gh, gl);
      sm.Gh[f * T::NN + slot] = gh;
      sm.Gl[f * T::NN + slot] = gl;
    }
    float c32;
    unsigned int okb = 0;
    if (cached) {
      c32 = a.node_c[idx];
      okb = a.node_ok[idx];
    } else {
      // FP32 sound speed: rho c^2 = gbar (p + pbar) (Sec. 2)
      const float a1 = vh[A] + vl[A];
      const float Gam32 = eos.r2f + eos.drf * a1;
      const float pb32 = __fdividef(eos.q1f * a1, Gam32 + 1.0f);
      const float rho32 = vh[0] + vh[1];
      const float pp = vh[E] + vl[E] + pb32;
      c32 = sqrtf(__fdividef((1.0f + __fdividef(1.0f, Gam32)) * pp, rho32));
      // Node quantities certified above the limiter tolerances (the first
      // test of Algorithms 1-3); bit set = certified.  hi is the value
      // truncated toward zero, so hi >= eps > 0 implies value >= eps.
      if (vh[0] >= epsf_ar) okb |= 1u;
      if (vh[1] >= epsf_ar) okb |= 2u;
      if (vh[A] >= epsf_a) okb |= 4u;
      if (((1.0f - vh[A]) - vl[A]) * (1.0f - 2.4e-7f) >= epsf_a) okb |= 8u;
      if (Gam32 * pp - margin(Gam32 * (fabsf(vh[E]) + pb32)) * 4.0f >= epsf_rc) okb |= 16u;
    }
    sm.c[slot] = c32;
    sm.ok[slot] = okb;
    if (DIR == FIRST && ln.valid && s >= 3 && s < 3 + T::TM - 1 && pos < n) {
      // input admissibility (Sec. 2), once per interior cell: 0 <= alpha1 <= 1
      // and the partial densities as integer compares of the bits; rho
      // ctilde^2 > 0 from the FP32 certification bit when it holds (it
      // certifies rho ctilde^2 >= eps_rc > 0), else from the FP64 value
      // multiplied through by Gamma + 1 > 0
      const bool adm = adm_ok && ((okb & 16u) || positive64(adm_rct));
      if (!adm) atomicAdd(&a.stats->inadmissible, 1ull);
    }
    // the first sweep fills the node cache for the cells its tile owns
    if (DIR == FIRST && a.node_write && ln.valid && s >= 3 && s < 3 + T::TM - 1 && pos < n) {
      a.node_p[idx] = p;
      a.node_ir[idx] = ir;
      a.node_c[idx] = c32;
      a.node_ok[idx] = okb;
    }
  }
  // block-wide scalars (dt, lambda_d of Sec. 3.3, combine coefficients),
  // computed once instead of by every thread: FP64 work is the scarce one
  if (tid == 0) {
    const double dt0 = geo.dt(), lam0 = geo.lam(), bdt0 = a.rk_b * dt0;
    sm.scal[0] = dt0;
    sm.scal[1] = lam0;
    sm.scal[2] = bdt0 * geo.l_unit();  // multiplies the L array (see SweepArgs::l_raw)
    sm.scal[3] = bdt0 * geo.inv_dx();
    reinterpret_cast<float *>(sm.scal + 4)[0] = (float)(2.0 * lam0);
    *sm.nslow = 0u;
  }
  __syncthreads();

  const double lam = sm.scal[1];
  const float l2 = reinterpret_cast<const float *>(sm.scal + 4)[0];
  const R epsR = a.eps_is32;
  const unsigned int ALL = 31u;

  // ---- 3: midpoint fluxes ---------------------------------------------------
  int nlim_i = 0, nhard_i = 0, nlim_f = 0, nhard_f = 0, nslow = 0;
  // One midpoint.  The fast instance (SLOW false) certifies both limiters
  // in FP32 and, where a certification fails, returns false without
  // writing anything; the slow instance computes those midpoints with the
  // FP64 limiter fallbacks.  Two instances keep the fallbacks' registers
  // out of the fast loop's allocation.
  auto midpoint = [&](const int q, auto slow_tag) -> bool {
    constexpr bool SLOW = decltype(slow_tag)::value;
    const int l = DIR == 0 ? q / T::TM : q % T::TL;
    const int m = DIR == 0 ? q % T::TM : q / T::TL;
    const int si = m + 2;
    const Line lnm = geo.line(l);
    const int cnt = (m < T::TM - 1 || tile0 + m == lnm.n) && tile0 + m <= lnm.n && lnm.valid;
    const int ni = nslot(l, si), ni1 = nslot(l, si + 1);
    // reference node i in FP32 (hi parts) and deviations of the stencil nodes
    float hi_i[NF], lo_i[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      hi_i[f] = sm.Vh[f * T::NN + ni];
      lo_i[f] = sm.Vl[f * T::NN + ni];
    }
    auto dev = [&](int s, float *d) {
      const int sl = nslot(l, s);
#pragma unroll
      for (int f = 0; f < NF; ++f) d[f] = (sm.Vh[f * T::NN + sl] - hi_i[f]) + (sm.Vl[f * T::NN + sl] - lo_i[f]);
    };
    auto gdev = [&](int s, int f) {
      const int sl = nslot(l, s);
      return (sm.Gh[f * T::NN + sl] - sm.Gh[f * T::NN + ni]) + (sm.Gl[f * T::NN + sl] - sm.Gl[f * T::NN + ni]);
    };
    RefNode<NDIM, R> ref;
    ref.r1 = hi_i[0];
    ref.r2 = hi_i[1];
    ref.rho = hi_i[0] + hi_i[1];
#pragma unroll
    for (int j = 0; j < NDIM; ++j) ref.u[j] = hi_i[2 + j];
    ref.p = hi_i[E];
    ref.a1 = hi_i[A];
    // FP32 conservative state of node nk from its primitive hi parts
    // (relative precision; used for (E + p)_ref and the half-state checks).
    auto wf_node = [&](int nk, float *Wo) {
      const float r1 = sm.Vh[0 * T::NN + nk], r2 = sm.Vh[1 * T::NN + nk], al = sm.Vh[A * T::NN + nk];
      const float pk = sm.Vh[E * T::NN + nk];
      const float rho = r1 + r2;
      float ke = 0.0f;
      Wo[0] = r1;
      Wo[1] = r2;
#pragma unroll
      for (int j = 0; j < NDIM; ++j) {
        const float u = sm.Vh[(2 + j) * T::NN + nk];
        Wo[2 + j] = rho * u;
        ke += u * u;
      }
      Wo[E] = pk * (eos.r2f + eos.drf * al) + eos.q1f * al + 0.5f * rho * ke;
      Wo[A] = al;
    };
    {
      float W0[NF];
      wf_node(ni, W0);
      ref.Ep = W0[E] + hi_i[E];
    }
    const float ci = sm.c[ni], ci1 = sm.c[ni1];

    // The high-order flux comes first; the first-order flux, the node states
    // and the node-flux deviations the certification needs are formed after
    // it, so that none of them is held in registers across WCNS-IS.
    float dGh[NF], duh;  // high-order G^ - G_i and u^ - u_i
    bool slow_flux = false;
    if (a.scheme != SCHEME_HLLC1) {
      const unsigned int ok_i = sm.ok[ni], ok_i1 = sm.ok[ni1];
      // Steps 1-2: projection with means of nodes i, i+1 (App. A).
      const float ar1 = 0.5f * (hi_i[0] + sm.Vh[0 * T::NN + ni1]);
      const float ar2 = 0.5f * (hi_i[1] + sm.Vh[1 * T::NN + ni1]);
      const float rb = ar1 + ar2;
      const float cb = 0.5f * (ci + ci1);
      const float irc = __fdividef(1.0f, rb * cb);
      const float k1 = ar1 * irc / cb, k2 = ar2 * irc / cb;
      // Steps 2-3 field by field: the projected deviations of two
      // characteristic fields at a time (stencil nodes j = 0..5 are
      // i-2..i+3; node i itself, j = 2, has zero deviation and enters
      // neither stencil of the deviation form) and their left / right
      // WCNS-IS interpolations (Sec. 4.3), so that only two fields'
      // stencils are held in registers at once.
      auto devc = [&](int j, int c) {
        const int sl = nslot(l, m + j);
        return (sm.Vh[c * T::NN + sl] - hi_i[c]) + (sm.Vl[c * T::NN + sl] - lo_i[c]);
      };
      float UL[NF], UR[NF];
      float dp[6];  // pressure deviations, shared by the three fields that involve p
#pragma unroll
      for (int j = 0; j < 6; ++j) dp[j] = j == 2 ? 0.0f : devc(j, E);
      {
        float a[6], b[6];
        // acoustic fields: 0 = (u_n - c), NF-1 = (u_n + c)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const float du = j == 2 ? 0.0f : devc(j, 2 + DIR);
          a[j] = du - irc * dp[j];
          b[j] = du + irc * dp[j];
        }
        UL[0] = wenois_c0<R>(a[0], a[1], a[3], a[4], epsR);
        UR[0] = wenois_p0<R>(a[5], a[4], a[3], a[1], epsR);
        UL[NF - 1] = wenois_c0<R>(b[0], b[1], b[3], b[4], epsR);
        UR[NF - 1] = wenois_p0<R>(b[5], b[4], b[3], b[1], epsR);
        // entropy / partial-density fields 1 and 2
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          a[j] = (j == 2 ? 0.0f : devc(j, 0)) - k1 * dp[j];
          b[j] = (j == 2 ? 0.0f : devc(j, 1)) - k2 * dp[j];
        }
        UL[1] = wenois_c0<R>(a[0], a[1], a[3], a[4], epsR);
        UR[1] = wenois_p0<R>(a[5], a[4], a[3], a[1], epsR);
        UL[2] = wenois_c0<R>(b[0], b[1], b[3], b[4], epsR);
        UR[2] = wenois_p0<R>(b[5], b[4], b[3], b[1], epsR);
        // tangential velocities and alpha1: plain deviations
        int row = 3;
#pragma unroll
        for (int k = 0; k <= NDIM; ++k) {
          if (k == DIR) continue;
          const int c = k < NDIM ? 2 + k : A;
          const int f = k < NDIM ? row++ : NF - 2;
#pragma unroll
          for (int j = 0; j < 6; ++j) a[j] = j == 2 ? 0.0f : devc(j, c);
          UL[f] = wenois_c0<R>(a[0], a[1], a[3], a[4], epsR);
          UR[f] = wenois_p0<R>(a[5], a[4], a[3], a[1], epsR);
        }
      }
      // Step 4: back-projection to primitive deviations.
      float dV[2][NF];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const float *Us = side ? UR : UL;
        float *d = dV[side];
        const float dac = Us[NF - 1] - Us[0];
        d[0] = Us[1] + __fdividef(ar1, 2.0f * cb) * dac;
        d[1] = Us[2] + __fdividef(ar2, 2.0f * cb) * dac;
        int row = 3;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
          if (k == DIR) {
            d[2 + k] = 0.5f * (Us[0] + Us[NF - 1]);
          } else {
            d[2 + k] = Us[row];
            ++row;
          }
        }
        d[E] = 0.5f * rb * cb * dac;
        d[A] = Us[NF - 2];
      }
      // Sound speeds of the interpolated states (Sec. 2), FP32.
      float cs[2];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const float *d = dV[side];
        const float a1 = ref.a1 + (lo_i[A] + d[A]);
        const float Gam = eos.r2f + eos.drf * a1;
        const float pb = __fdividef(eos.q1f * a1, Gam + 1.0f);
        const float rho = ref.rho + (lo_i[0] + lo_i[1] + d[0] + d[1]);
        cs[side] = sqrtf(__fdividef((1.0f + __fdividef(1.0f, Gam)) * (ref.p + (lo_i[E] + d[E]) + pb), rho));
      }
      // Interpolation limiter (Sec. 5.1): FP32 certification, else FP64.
      if (a.scheme == SCHEME_PP) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          float *d = dV[side];
          const unsigned int okn = side ? ok_i1 : ok_i;
          bool cert = okn == ALL;
          if (cert) {
            const float r1 = hi_i[0] + (lo_i[0] + d[0]);
            const float r2 = hi_i[1] + (lo_i[1] + d[1]);
            const float al = hi_i[A] + (lo_i[A] + d[A]);
            const float om = ((1.0f - hi_i[A]) - lo_i[A]) - d[A];
            const float pt = hi_i[E] + (lo_i[E] + d[E]);
            const float Gam = eos.r2f + eos.drf * al;
            const float pb = __fdividef(eos.q1f * al, Gam + 1.0f);
            cert = r1 - margin(fabsf(hi_i[0]) + fabsf(d[0])) >= epsf_ar &&
                   r2 - margin(fabsf(hi_i[1]) + fabsf(d[1])) >= epsf_ar &&
                   al - margin(fabsf(hi_i[A]) + fabsf(d[A])) >= epsf_a &&
                   om - margin(fabsf(om) + fabsf(d[A])) >= epsf_a &&
                   Gam * (pt + pb) - margin(Gam * (fabsf(hi_i[E]) + fabsf(d[E]) + pb)) * 4.0f >= epsf_rc;
          }
          if (cert) continue;
          if constexpr (!SLOW) return false;
          nslow += cnt;
          FVec<NF> hv, lv, dv;
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            hv.v[f] = hi_i[f];
            lv.v[f] = lo_i[f];
            dv.v[f] = d[f];
          }
          const LimitedState<NF> ls =
              mixed_interp_fallback<NDIM>(eos, tol, sm.W, T::NN, side ? ni1 : ni, hv, lv, dv);
          nlim_i += cnt * (ls.flags & 1);
          nhard_i += cnt * (ls.flags >> 1);
          if (ls.flags) {
#pragma unroll
            for (int f = 0; f < NF; ++f) d[f] = ls.d[f];
            cs[side] = ls.c;
          }
        }
      }
      // Steps 6-8: midpoint HLLC and HCS reconstruction, deviation form.
      float dGt[NF], ut;
      hllc_dev<NDIM, DIR, R>(ref, eos, dV[0], cs[0], dV[1], cs[1], dGt, ut);
#pragma unroll
      for (int f = 0; f < NF; ++f)
        dGh[f] = hcs<R>(dGt[f], gdev(m, f), gdev(m + 1, f), 0.0f, gdev(si + 1, f), gdev(m + 4, f),
                        gdev(m + 5, f));
      {
        auto udev = [&](int s) {
          const int sl = nslot(l, s);
          return (sm.Vh[(2 + DIR) * T::NN + sl] - hi_i[2 + DIR]) + (sm.Vl[(2 + DIR) * T::NN + sl] - lo_i[2 + DIR]);
        };
        duh = hcs<R>(ut - ref.u[DIR] - lo_i[2 + DIR], udev(m), udev(m + 1), 0.0f, udev(m + 3), udev(m + 4),
                     udev(m + 5));
      }
    }
    // First-order HLLC in deviation form (Sec. 3.2).
    float d1[NF];  // node i+1
    dev(si + 1, d1);
    float dGH[NF], sH;
    {
      float d0[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) d0[f] = 0.0f;
      hllc_dev<NDIM, DIR, R>(ref, eos, d0, ci, d1, ci1, dGH, sH);
    }
    if (a.scheme == SCHEME_HLLC1) {
#pragma unroll
      for (int f = 0; f < NF; ++f) dGh[f] = dGH[f];
      duh = sH - ref.u[DIR];
    }
    // Delta of alpha between the nodes, node states and node-flux deviation
    // of node i+1 for the flux-limiter certification
    const float dal = d1[A];
    const unsigned int ok_i = sm.ok[ni], ok_i1 = sm.ok[ni1];
    float Wf[2][NF];
    wf_node(ni, Wf[0]);
    wf_node(ni1, Wf[1]);
    float dG1[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) dG1[f] = gdev(si + 1, f);
    // alpha1 components of the split high-order flux (Sec. 3.2), evaluated
    // once: the certification below tests the very values the update applies.
    const float ai = hi_i[A], ai1 = hi_i[A] + dal, ui = ref.u[DIR];
    const float gmA = dGh[A] - ai * duh;
    const float gpA = (ai - ai1) * ui + dGh[A] - ai1 * duh;
    // Flux limiter (Sec. 5.2): FP32 certification that every quantity of the
    // four half states is at least its tolerance (then every theta is 1).
    // margin() is taken over the operands' magnitudes, so cancellation in a
    // difference is covered; |G_i| 2^-26 covers the rounding of the FP32
    // node-flux deviations and of G_i + dG in FP64.
    if (a.scheme == SCHEME_PP) {
      bool cert = ok_i == ALL && ok_i1 == ALL;
#pragma unroll
      for (int st = 0; st < 4; ++st) {
        if (!cert) break;
        // st: 0 = W_i^{HLLC,+}, 1 = W_{i+1}^{HLLC,-}, 2 = W_i^{+}, 3 = W_{i+1}^{-}
        const bool hl = st < 2;
        const bool right = st & 1;
        const float *dg = hl ? dGH : dGh;
        const float sgn = right ? 1.0f : -1.0f;  // W_i - 2 lam (.), W_{i+1} + 2 lam (.)
        const float *wn = Wf[right ? 1 : 0];
        float x[NF], mag[NF];
#pragma unroll
        for (int f = 0; f < NF - 1; ++f) {
          const float D = right ? dg[f] - dG1[f] : dg[f];
          const float ops = fabsf(dg[f]) + (right ? fabsf(dG1[f]) : 0.0f) + 1.5e-8f * fabsf(sm.Gh[f * T::NN + ni]);
          x[f] = wn[f] + sgn * l2 * D;
          mag[f] = fabsf(wn[f]) + l2 * ops;
        }
        float DA, opsA;
        if (hl) {
          const float du = sH - ui - lo_i[2 + DIR];
          DA = right ? -dal * ui + dg[A] - ai1 * du : dg[A] - ai * du;
          opsA = fabsf(dg[A]) + fabsf((right ? ai1 : ai) * du) + (right ? fabsf(dal * ui) : 0.0f);
        } else {
          DA = right ? gpA : gmA;
          opsA = fabsf(DA);
        }
        x[A] = wn[A] + sgn * l2 * DA;
        mag[A] = fabsf(wn[A]) + l2 * opsA;
        // 1 - alpha of the node from its hi/lo parts, then the step
        const float omn = right ? ((1.0f - hi_i[A]) - lo_i[A]) - dal : (1.0f - hi_i[A]) - lo_i[A];
        const float om = omn - sgn * l2 * DA;
        cert = x[0] - margin(mag[0]) >= epsf_ar && x[1] - margin(mag[1]) >= epsf_ar &&
               x[A] - margin(mag[A]) >= epsf_a && om - margin(fabsf(omn) + fabsf(dal) + l2 * opsA) >= epsf_a &&
               rct2_certified<NDIM>(eos, x, mag, epsf_rc);
      }
      slow_flux = !cert;
      if constexpr (!SLOW) {
        if (slow_flux) return false;
      }
      nslow += cnt * (int)slow_flux;
    }
    // Assemble the FP64 split fluxes G^-_{i+1/2}, G^+_{i+1/2} (Sec. 3.2).
    const int ms = mslot(l, m);
    if (!slow_flux) {
#pragma unroll
      for (int f = 0; f < NF - 1; ++f) sm.F[f * T::NM + ms] = sm.G[f * T::NN + ni] + f2d(dGh[f]);
      sm.am[ms] = f2d(gmA);
      sm.ap[ms] = f2d(gpA);
    } else {
      FVec<NF> dgv;
#pragma unroll
      for (int f = 0; f < NF; ++f) dgv.v[f] = dGh[f];
      const double ui64 = (double)hi_i[2 + DIR] + (double)lo_i[2 + DIR];
      const int fl = mixed_flux_fallback<NDIM, DIR>(eos, tol, sm.W, sm.G, T::NN, ni, ni1, sm.F, sm.am, sm.ap,
                                                    T::NM, ms, ui64, duh, dgv, lam);
      nlim_f += cnt * (fl & 1);
      nhard_f += cnt * (fl >> 1);
    }
    return true;
  };
  bool barrier_done = false;
  if constexpr (DEFER) {
    int deferred = 0;
    for (int q = tid; q < T::NM; q += T::THREADS)
      if (!midpoint(q, std::false_type{})) {
        sm.slow[atomicAdd(sm.nslow, 1u)] = q;
        deferred = 1;
      }
    // one barrier when nothing was deferred (it also orders the flux
    // stores before the cell update); the second pass only when needed
    if (__syncthreads_or(deferred)) {
      const int nsl = (int)*sm.nslow;
      for (int k = tid; k < nsl; k += T::THREADS) midpoint(sm.slow[k], std::true_type{});
    } else {
      barrier_done = true;
    }
  } else {
    for (int q = tid; q < T::NM; q += T::THREADS) midpoint(q, std::true_type{});
  }
  if (nlim_i) atomicAdd(&a.stats->interp_limited, (unsigned long long)nlim_i);
  if (nhard_i) atomicAdd(&a.stats->interp_hard, (unsigned long long)nhard_i);
  if (nlim_f) atomicAdd(&a.stats->flux_limited, (unsigned long long)nlim_f);
  if (nhard_f) atomicAdd(&a.stats->flux_hard, (unsigned long long)nhard_f);
  if (nslow) atomicAdd(&a.stats->fp64_fallbacks, (unsigned long long)nslow);
  if (!barrier_done) __syncthreads();

  // ---- 4: cell update (FP64) -------------------------------------------------
  float smax_local[NDIM];
#pragma unroll
  for (int j = 0; j < NDIM; ++j) smax_local[j] = 0.0f;
  int done = 0;
  const double idx_ = geo.inv_dx();
  const double bdt = sm.scal[2], bdt_idx = sm.scal[3];
  // stage 1 of SSPRK3 has b = 1 and a = 0: skip those FP64 operations
  // (tested on the bit patterns: integer compares, not the FP64 pipe)
  const bool b_one = __double_as_longlong(a.rk_b) == 0x3FF0000000000000ll;
  const bool has_a = (__double_as_longlong(a.rk_a) << 1) != 0;
  for (int q = tid; q < T::TL * (T::TM - 1); q += T::THREADS) {
    const int l = DIR == 0 ? q / (T::TM - 1) : q % T::TL;
    const int m = DIR == 0 ? q % (T::TM - 1) : q / T::TL;
    const Line ln = geo.line(l);
    const int pos = tile0 + m;
    if (!ln.valid || pos >= ln.n) continue;
    ++done;
    const long long idx = ln.base + (long long)pos * ln.stride;
    const int ml = mslot(l, m), mr = mslot(l, m + 1);
    if (a.epilogue != EPI_COMBINE) {
      double diff[NF];
#pragma unroll
      for (int f = 0; f < NF - 1; ++f) diff[f] = sm.F[f * T::NM + ml] - sm.F[f * T::NM + mr];
      diff[A] = sm.ap[ml] - sm.am[mr];
      if (a.epilogue == EPI_WRITE) {
        // inside a step the raw difference; the combine applies 1/dx
#pragma unroll
        for (int f = 0; f < NF; ++f) a.L[(long long)f * N + idx] = a.l_raw ? diff[f] : diff[f] * idx_;
      } else {
        // every load of the cell before its stores: the compiler cannot tell
        // the components apart, and would order each load after the last store
        double l0[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) l0[f] = a.L[(long long)f * N + idx];
#pragma unroll
        for (int f = 0; f < NF; ++f) a.L[(long long)f * N + idx] = fma(diff[f], geo.accum_scale(), l0[f]);
      }
    } else {
      const int ns = nslot(l, m + 3);
      double w[NF], wn[NF], lv[NF];
      bool finite = true;
      // loads first, as above (W_out may be any other array)
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        wn[f] = has_a ? a.Wn[(long long)f * N + idx] : 0.0;
        lv[f] = a.read_L ? a.L[(long long)f * N + idx] : 0.0;
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        // a W^n + b W + b dt (L + flux difference / dx) (Sec. 5.3 combine)
        const double diff = f < NF - 1 ? sm.F[f * T::NM + ml] - sm.F[f * T::NM + mr] : sm.ap[ml] - sm.am[mr];
        const double wi = sm.W[f * T::NN + ns];
        double acc = b_one ? wi : a.rk_b * wi;
        if (has_a) acc = fma(a.rk_a, wn[f], acc);
        if (a.read_L) acc = fma(bdt, lv[f], acc);
        w[f] = fma(bdt_idx, diff, acc);
        finite = finite && finite64(w[f]);
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) a.W_out[(long long)f * N + idx] = w[f];
      if (!finite) atomicAdd(&a.stats->nonfinite, 1ull);
      // max(|u_d| + c) of the new state for the next stage (FP32 suffices
      // for the directional split, Sec. 3.3)
      float hi, lo;
      float wf[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        split_hilo(w[f], hi, lo);
        wf[f] = hi + lo;
      }
      const float rho = wf[0] + wf[1];
      float m2 = 0.0f;
#pragma unroll
      for (int j = 0; j < NDIM; ++j) m2 += wf[2 + j] * wf[2 + j];
      const float Gam = eos.r2f + eos.drf * wf[A];
      const float pb = __fdividef(eos.q1f * wf[A], Gam + 1.0f);
      const float ke = 0.5f * __fdividef(m2, rho);
      // rho ctilde^2 = E - ke - pbar loses digits to cancellation when the
      // kinetic energy dominates: take it plus its FP32 error bound
      // (8 2^-24 of the terms' magnitudes), so that c, and the wave speed
      // that sets the next stage's lambda (Sec. 3.3), is never underestimated
      const float rct = (wf[E] - ke - pb) + 4.76837158203125e-07f * (fabsf(wf[E]) + ke + pb);
      const float iG = __fdividef(1.0f, Gam);
      const float c = sqrtf(fmaxf((1.0f + iG) * iG * rct, 0.0f) / rho);
#pragma unroll
      for (int j = 0; j < NDIM; ++j) {
        const float sj = fabsf(__fdividef(wf[2 + j], rho)) + c;
        smax_local[j] = (sj > smax_local[j] || sj != sj) ? sj : smax_local[j];
      }
    }
  }
  if (a.epilogue == EPI_COMBINE) {
#pragma unroll
    for (int j = 0; j < NDIM; ++j) {
      // the warp's maximum on the FP32 bit patterns (non-negative floats
      // and NaNs order like their bits), then one conversion with 1 + 2^-20
      // headroom, so that the FP32 maximum never undercuts the FP64 one
      const unsigned int fb = __reduce_max_sync(0xffffffffu, __float_as_uint(smax_local[j]));
      if ((tid & 31) == 0 && fb) {
        const double m = (double)__uint_as_float(fb) * (1.0 + 9.5367431640625e-07);
        atomicMax(geo.smax_slot(j), (unsigned long long)__double_as_longlong(m));
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) done += __shfl_xor_sync(0xffffffffu, done, o);
  if ((tid & 31) == 0 && done) atomicAdd(&a.stats->midpoints, (unsigned long long)done);
}

template <int NDIM, int DIR, class T>
__global__ void __launch_bounds__(T::THREADS,
                                  NDIM == 2 ? MIXED_MIN_BLOCKS_2D
                                            : (NDIM == 3 ? (T::THREADS <= 128 ? 8 : MIXED_MIN_BLOCKS_3D)
                                                         : MIXED_MIN_BLOCKS))
    sweep_kernel_mixed(const SweepArgs a) {
  extern __shared__ double smem_raw[];
  if (!a.ctl->active) return;
  sweep_body_mixed<NDIM, DIR, T>(a, GridGeo<NDIM, DIR, T>(a), smem_raw);
}

template <int NDIM, int DIR, class T = TileMixed<NDIM, DIR>>
cudaError_t launch_sweep_mixed_t(const SweepArgs &a, cudaStream_t st) {
  const size_t bytes = SmemMixed<NDIM, T>::BYTES;
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = configure_once(configured, [&] {
    cudaError_t r = cudaFuncSetAttribute(sweep_kernel_mixed<NDIM, DIR, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(sweep_kernel_mixed<NDIM, DIR, T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               100);
    return r;
  });
  if (e != cudaSuccess) return e;
  sweep_kernel_mixed<NDIM, DIR, T><<<sweep_grid<DIR, T>(a), T::THREADS, bytes, st>>>(a);
  return cudaGetLastError();
}


}  // namespace wcns
