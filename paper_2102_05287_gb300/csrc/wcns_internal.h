// Internal declarations shared by the CUDA translation units of libwcns.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace wcns {

// One-time configuration of a kernel's function attributes, which CUDA
// keeps per device: `once` holds one bit per device ordinal (ordinals of 64
// and above configure on every call).
template <class F>
inline cudaError_t configure_once(std::atomic<unsigned long long> &once, F &&configure) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (once.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = configure();
  if (e == cudaSuccess && bit) once.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}


// Per-phase EOS constants (Sec. 2): with Gamma(a1) = 1/(gbar-1) and
// Pi(a1) = gbar pbar/(gbar-1),
//   Gamma = a1 * r1 + (1 - a1) * r2,   Pi = a1 * q1   (the gas has pinf = 0).
struct EosConst {
  double r1;  // 1/(gamma_l - 1)
  double r2;  // 1/(gamma_g - 1)
  double q1;  // gamma_l pinf_l / (gamma_l - 1)
  double dr;  // r1 - r2
  float r2f, drf, q1f;  // FP32 copies for the mixed path, rounded once here
};

inline EosConst make_eos(double gamma_g, double gamma_l, double pinf_l) {
  EosConst e;
  e.r1 = 1.0 / (gamma_l - 1.0);
  e.r2 = 1.0 / (gamma_g - 1.0);
  e.q1 = gamma_l * pinf_l / (gamma_l - 1.0);
  e.dr = e.r1 - e.r2;
  e.r2f = (float)e.r2;
  e.drf = (float)e.dr;
  e.q1f = (float)e.q1;
  return e;
}

struct LimTol {
  double eps_ar, eps_a, eps_rc;  // Algorithms 1-6 tolerances
  double hs_ar, hs_a, hs_rc;     // hard-switch tolerances
  // FP32 certification thresholds of the mixed path: eps (1 + 1e-6) rounded
  // to FP32, so "x >= cert" implies "x >= eps"
  float cert_ar, cert_a, cert_rc;
  // every hard-switch tolerance <= its limiter tolerance: then a state that
  // passed all threshold tests unblended cannot fail a hard-switch test
  int hs_implied;
};

// Limiter and hard-switch tolerances must be finite and >= 0 (the kernels
// compare against them as bit patterns), the IS epsilon finite and > 0.
template <class Options>
inline bool valid_tolerances(const Options &o) {
  const double v[6] = {o.eps_ar, o.eps_a, o.eps_rc, o.hs_ar, o.hs_a, o.hs_rc};
  for (double x : v)
    if (!(x >= 0.0) || !(x < 1e300)) return false;
  return o.eps_is > 0.0 && o.eps_is < 1e300;
}

inline void set_cert(LimTol &t) {
  t.cert_ar = (float)(t.eps_ar * (1.0 + 1e-6));
  t.cert_a = (float)(t.eps_a * (1.0 + 1e-6));
  t.cert_rc = (float)(t.eps_rc * (1.0 + 1e-6));
  t.hs_implied = t.hs_ar <= t.eps_ar && t.hs_a <= t.eps_a && t.hs_rc <= t.eps_rc;
}

// Device counters (accumulated with integer atomics: order-independent).
struct DevStats {
  unsigned long long interp_limited;
  unsigned long long interp_hard;
  unsigned long long flux_limited;
  unsigned long long flux_hard;
  unsigned long long nonfinite;
  unsigned long long inadmissible;
  unsigned long long midpoints;
  unsigned long long fp64_fallbacks;  // mixed path: limiter work not certified in FP32
};

// Time-step control kept in device memory so that whole steps can run (and
// be captured in a CUDA graph) without host round trips.
//   smax[k][d]: bit patterns of max(|u_d| + c) of stage-input state k
//   (k = 0: W^n, 1: W^(1), 2: W^(2), 3: W^(n+1)); non-negative doubles
//   order like their bit patterns, so atomicMax on the bits is exact.
struct StepCtl {
  unsigned long long smax[4][3];
  unsigned long long smax_bc[3];  // max(|u_d| + c) of the Dirichlet ghost states: the
                                  // floor every wave-speed slot starts from
  double dt;        // step size of the current step
  double t;         // time after the current step
  double t_end;     // advance-to target (or +inf)
  long long steps;  // steps taken
  int active;       // 0 once t has reached t_end: remaining kernels do nothing
  // DevStats inadmissible / nonfinite counts when the current call began:
  // a synchronising call compares them with the counts at its end
  unsigned long long stat0[2];
};

// Status of the work enqueued since the counters were snapshotted into
// stat0: a non-finite update first, then a stage input outside G (Sec. 2).
inline int status_from_counts(const StepCtl &c, const DevStats &s, int ok, int e_nonfinite, int e_inadmissible) {
  if (s.nonfinite > c.stat0[1]) return e_nonfinite;
  if (s.inadmissible > c.stat0[0]) return e_inadmissible;
  return ok;
}

#ifdef __CUDACC__
// |u_d| + c of one conservative state for d < ndim (Sec. 3.3), with the FP64
// mixture thermodynamics of Sec. 2: p = (rho e - Pi)/Gamma,
// pbar = Pi/(Gamma + 1), rho c^2 = (1 + 1/Gamma)(p + pbar).  Every FP64
// reduction of max(|u_d| + c) (single grids, Dirichlet states, batched
// problems) uses this one function, so that they agree bit for bit.
__device__ __forceinline__ void state_wavespeeds(double a1r1, double a2r2, const double *m, double E, double a1,
                                                 int ndim, const EosConst &e, double *s) {
  const double rho = a1r1 + a2r2;
  const double ir = 1.0 / rho;
  double m2 = 0.0, v[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < ndim; ++j) {
    v[j] = m[j] * ir;
    m2 = fma(m[j], v[j], m2);
  }
  const double rhoe = E - 0.5 * m2;
  const double Gam = fma(a1, e.r1 - e.r2, e.r2);
  const double Pi = a1 * e.q1;
  const double iG = 1.0 / Gam;
  const double p = (rhoe - Pi) * iG;
  const double pb = Pi / (Gam + 1.0);
  const double c = sqrt((1.0 + iG) * (p + pb) * ir);
  for (int j = 0; j < ndim; ++j) s[j] = fabs(v[j]) + c;
}
#endif

// Order of the directional sweeps of one mixed-precision RHS evaluation:
// with MIXED_REVERSE_SWEEPS the last axis goes first and x last, so that
// the sweep that carries the SSPRK3 combine (its extra W^n and L reads and
// the state write) is the x sweep, whose tiles read and write whole rows.
// The first sweep of an RHS fills the node cache and counts inadmissible
// inputs; the FP64 path keeps the order x, y, z.
#ifndef MIXED_REVERSE_SWEEPS
#define MIXED_REVERSE_SWEEPS 1
#endif
__host__ __device__ constexpr int mixed_first_dir(int ndim) { return MIXED_REVERSE_SWEEPS ? ndim - 1 : 0; }

enum Epilogue {
  EPI_WRITE = 0,     // L  = contribution
  EPI_ACCUM = 1,     // L += contribution
  EPI_COMBINE = 2,   // W_out = a W^n + b (W_in + dt (L? + contribution)), plus wave-speed max
};

enum { SCHEME_PP = 0, SCHEME_HLLC1 = 1, SCHEME_WCNS = 2 };
enum { BC_TRANS = 0, BC_PERIODIC = 1, BC_SYMMETRY = 2, BC_DIRICHLET = 3 };

struct SweepArgs {
  int n[3];                 // cells per axis (1 beyond ndim)
  long long ncell;          // product of n
  int bc_lo, bc_hi;         // boundary kinds of the swept axis
  double dir_lo[7], dir_hi[7];  // Dirichlet ghost states of the swept axis
  const double *dir_face_lo;    // optional per-face Dirichlet states [nf][face_n]
  const double *dir_face_hi;    //   (NULL: dir_lo / dir_hi on the whole face)
  long long face_n;             // cells on a face normal to the swept axis
  double inv_dx;            // 1/dx of the swept axis
  double inv_dx_all[3];     // 1/dx of every axis
  EosConst eos;
  LimTol tol;
  double eps_is;
  float eps_is32;           // max(eps_is, 1e-30) in FP32 (mixed path)
  int scheme;
  int epilogue;
  int read_L;               // EPI_COMBINE: add the L array (earlier directions)
  double rk_a, rk_b;        // combine coefficients
  int stage;                // 0, 1, 2: lambda from ctl->smax[stage]; the combine
                            // epilogue reduces into ctl->smax[stage + 1]
  // Mixed path, 2D/3D: node quantities shared by the sweeps of one RHS
  // evaluation (all sweeps read the same stage input).  The first sweep
  // stores, for every cell it owns, p and 1/rho (FP64), the FP32 sound
  // speed and the certification bits; the later sweeps load them for every
  // node that is a cell or a copy of one (Dirichlet ghosts are computed).
  double *node_p, *node_ir;
  float *node_c;
  unsigned int *node_ok;
  int node_write, node_read;
  // Scaling of the L array (mixed path): with l_raw = 1 (inside a step)
  // the first sweep stores its flux difference without the 1/dx factor,
  // later sweeps add diff * accum_scale (= inv_dx_d / inv_dx_0) and the
  // combine multiplies L by l_unit (= inv_dx_0).  Otherwise l_raw = 0,
  // accum_scale = inv_dx_d and l_unit = 1: L is the right-hand side itself.
  int l_raw;
  double accum_scale;
  double l_unit;
  const double *W_in;       // stage input state
  const double *Wn;         // W^n (combine with rk_a != 0)
  double *W_out;            // combine output
  double *L;                // RHS accumulator
  StepCtl *ctl;             // device step control (dt, wave-speed maxima)
  DevStats *stats;
};

// Launchers (defined per precision in wcns_fp64.cu / wcns_mixed.cu).
cudaError_t launch_sweep_fp64(int ndim, int dir, const SweepArgs &a, cudaStream_t s);
cudaError_t launch_sweep_mixed(int ndim, int dir, const SweepArgs &a, cudaStream_t s);

}  // namespace wcns
