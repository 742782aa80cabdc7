// Plain FP64 CPU oracle for the PP-WCNS-IS right-hand side of the
// five-equation (Allaire) two-phase model, following Wong, Angel, Barad &
// Kiris, "A positivity-preserving high-order weighted compact nonlinear
// scheme for compressible gas-liquid flows" (arXiv 2102.05287).
//
// TEST INFRASTRUCTURE.  This file is the parity reference for the CUDA
// library and the timed CPU baseline.  Only the test-suite, the smoke check,
// the benchmark's CPU-baseline legs and reference arm, and opcount_table.py
// load it.  It shares no code, header, table or constant with the CUDA path.
//
// Style: scalar loops, no fusion, one step of the paper per function, in the
// paper's order and notation.  Build with -O2 -ffp-contract=off so every
// product and sum is rounded as written.  Compiling with -DORACLE_COUNT_OPS
// turns `real` into an operation-counting scalar (opcount.hpp) that yields
// the algorithmic operation mix of one RHS evaluation.
//
// Phase 1 is the liquid (stiffened gas, gamma_l, pinf_l), phase 2 the gas
// (ideal, gamma_g, pinf = 0), as in the paper's fluid table (Section 6).
//
// Conservative vector per cell (Section 2):
//   W = (a1r1, a2r2, rho*u_1 .. rho*u_ndim, E, alpha1),  nf = ndim + 4.
// Primitive vector (Appendix A):
//   V = (a1r1, a2r2, u_1 .. u_ndim, p, alpha1).
// Both use the same slot positions.
//
// Readings of the paper where it is silent (each also listed in the design
// notes):
//   * epsilon of the IS weights is a parameter (default 1e-40);
//   * sign(0) = 0 in the HLLC flux (Section 3.2, as written);
//   * the projection matrices at i+1/2 use arithmetic means of a1r1, a2r2,
//     rho (sum of the two means) and c of nodes i and i+1 (Section 4.2);
//   * the flux-limiter half states use the physical flux F (zero alpha
//     component), Section 5.2;
//   * lambda_d = dt / (dx_d * sigma_d) with sigma_d from the state passed to
//     the RHS (Section 3.3), so sigma = 1 and lambda = dt/dx in 1D;
//   * three ghost layers per side: transmissive = zero-gradient copy,
//     periodic = wrap, symmetry = mirror with the normal momentum negated,
//     Dirichlet = a fixed conservative state;
//   * SSPRK3 is the Shu-Osher three-stage form (Section 5.3 cites it).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

// Steps of the method, for the op-counting build's per-step tallies.
enum OcRow {
  ROW_OTHER = 0,
  ROW_NODE_EOS = 2,      // node primitives: velocities, p, c (Section 2)
  ROW_PROJECT = 3,       // characteristic projection (Appendix A)
  ROW_WCNS_IS = 4,       // WCNS-IS interpolation (Section 4.3)
  ROW_BACKPROJECT = 5,   // back-projection and V -> W (Section 4.2)
  ROW_INTERP_LIMIT = 6,  // interpolation limiter (Section 5.1)
  ROW_MID_HLLC = 7,      // midpoint HLLC flux (Sections 3.1-3.2)
  ROW_NODE_FLUX = 8,     // node fluxes G_j (Section 4.2, step 7)
  ROW_HCS = 9,           // HCS reconstruction and the split (Sections 4.1, 3.2)
  ROW_HLLC1 = 10,        // first-order HLLC flux and its split (Section 3.2)
  ROW_FLUX_LIMIT = 11,   // flux limiter (Section 5.2)
  ROW_UPDATE = 12,       // flux difference + alpha1 div u (Section 4)
  ROW_WAVESPEED = 13,    // maximum wave speed (Section 3.3)
  ROW_COMBINE = 14,      // SSPRK3 stage combination (Section 5.3)
};

#ifdef ORACLE_COUNT_OPS
#include "opcount.hpp"
OracleOpCounts g_oracle_ops = {0, 0, 0, 0, 0};
OracleOpCounts g_oracle_rows[ORACLE_NROWS] = {};
int g_oracle_row = ROW_OTHER;
#define OC_ROW(r) (g_oracle_row = (r))
typedef Counted real;
#else
#define OC_ROW(r) ((void)0)
typedef double real;
static inline real o_sqrt(real a) { return std::sqrt(a); }
static inline real o_min(real a, real b) { return a < b ? a : b; }
static inline real o_max(real a, real b) { return a > b ? a : b; }
static inline real o_abs(real a) { return std::fabs(a); }
static inline double o_val(real a) { return a; }
static inline bool o_isfinite(real a) { return std::isfinite(a); }
#endif

extern "C" {

// Boundary kinds.
enum { OC_BC_TRANSMISSIVE = 0, OC_BC_PERIODIC = 1, OC_BC_SYMMETRY = 2, OC_BC_DIRICHLET = 3 };
// Schemes: the paper's PP-WCNS-IS, the first-order HLLC scheme of Section 3,
// and WCNS-IS with both limiters switched off.
enum { OC_SCHEME_PP_WCNS_IS = 0, OC_SCHEME_HLLC1 = 1, OC_SCHEME_WCNS_IS = 2 };

typedef struct {
  int ndim;
  int n[3];
  double lo[3], hi[3];
  int bc[3][2];
  double dirichlet[3][2][7];  // conservative ghost state for Dirichlet faces
  double gamma_g, gamma_l, pinf_l;
  int scheme;
  double eps_is;                 // epsilon of the IS nonlinear weights
  double eps_ar, eps_a, eps_rc;  // limiter tolerances (Section 5.1)
  double hs_ar, hs_a, hs_rc;     // hard-switch tolerances (Section 5.1)
  // Optional per-face Dirichlet states: dir_face[d][side] = NULL (use
  // dirichlet[d][side] everywhere) or [nf][face cells], the face cells
  // ordered by the other axes in increasing order, the lower one fastest.
  const double *dir_face[3][2];
} oc_config;

typedef struct {
  long long interp_limited;   // left/right interpolated states with some theta < 1
  long long interp_hard;      // interpolation hard switches
  long long flux_limited;     // midpoints with some flux-limiter theta < 1
  long long flux_hard;        // flux hard switches
  long long midpoints;        // midpoints evaluated
} oc_stats;

}  // extern "C"

namespace {

// ---------------------------------------------------------------------------
// Section 2: equation of state and mixture rules.
// ---------------------------------------------------------------------------
struct Eos {
  double g1, p1;  // phase 1: liquid (stiffened gas)
  double g2, p2;  // phase 2: gas (ideal, p2 = 0)
  // Per-phase constants 1/(g_k-1) and g_k p_k/(g_k-1).
  double r1, r2, q1, q2;
};

// Gamma(a1) := 1/(gbar-1) = a1/(g1-1) + a2/(g2-1)
static real mix_Gamma(const Eos &e, real a1) {
  real a2 = 1.0 - a1;
  return a1 * e.r1 + a2 * e.r2;
}
// Pi(a1) := gbar*pbar/(gbar-1) = a1*g1*p1/(g1-1) + a2*g2*p2/(g2-1)
static real mix_Pi(const Eos &e, real a1) {
  real a2 = 1.0 - a1;
  return a1 * e.q1 + a2 * e.q2;
}
// gbar = 1 + 1/Gamma and pbar = Pi (gbar-1)/gbar, from the two relations above.
static real mix_gamma(const Eos &e, real a1) { return 1.0 + 1.0 / mix_Gamma(e, a1); }
static real mix_pinf(const Eos &e, real a1) {
  real gb = mix_gamma(e, a1);
  return mix_Pi(e, a1) * (gb - 1.0) / gb;
}

struct Thermo {
  real rho, rhoe, p, rho_c2, rho_ct2, c;
  real vel[3];
};

// Mixture thermodynamics of a conservative state (Section 2):
//   p/(gbar-1) + gbar pbar/(gbar-1) = rho e,
//   rho c^2 = gbar (p + pbar),  rho ctilde^2 = rho e - pbar.
static Thermo thermo(const Eos &e, int ndim, const real *W) {
  Thermo t;
  int E = 2 + ndim, A = 3 + ndim;
  t.rho = W[0] + W[1];
  real ke = 0.0;
  for (int j = 0; j < ndim; ++j) {
    t.vel[j] = W[2 + j] / t.rho;
    ke = ke + W[2 + j] * W[2 + j];
  }
  t.rhoe = W[E] - 0.5 * ke / t.rho;
  t.p = (t.rhoe - mix_Pi(e, W[A])) / mix_Gamma(e, W[A]);
  real gb = mix_gamma(e, W[A]);
  real pb = mix_pinf(e, W[A]);
  t.rho_c2 = gb * (t.p + pb);
  t.rho_ct2 = t.rhoe - pb;
  t.c = o_sqrt(t.rho_c2 / t.rho);
  return t;
}

// rho*ctilde^2 = rho e - pbar_inf (Section 5.1 helper); same arithmetic as
// in thermo().
static real rho_ct2_of(const Eos &e, int ndim, const real *W) {
  int E = 2 + ndim, A = 3 + ndim;
  real rho = W[0] + W[1];
  real ke = 0.0;
  for (int j = 0; j < ndim; ++j) ke = ke + W[2 + j] * W[2 + j];
  real rhoe = W[E] - 0.5 * ke / rho;
  return rhoe - mix_pinf(e, W[A]);
}

static void cons_to_prim(const Eos &e, int ndim, const real *W, real *V) {
  Thermo t = thermo(e, ndim, W);
  V[0] = W[0];
  V[1] = W[1];
  for (int j = 0; j < ndim; ++j) V[2 + j] = t.vel[j];
  V[2 + ndim] = t.p;
  V[3 + ndim] = W[3 + ndim];
}

static void prim_to_cons(const Eos &e, int ndim, const real *V, real *W) {
  real rho = V[0] + V[1];
  real a1 = V[3 + ndim];
  real p = V[2 + ndim];
  // rho e = p/(gbar-1) + gbar*pbar/(gbar-1)
  real rhoe = p * mix_Gamma(e, a1) + mix_Pi(e, a1);
  real ke = 0.0;
  W[0] = V[0];
  W[1] = V[1];
  for (int j = 0; j < ndim; ++j) {
    W[2 + j] = rho * V[2 + j];
    ke = ke + V[2 + j] * V[2 + j];
  }
  W[2 + ndim] = rhoe + 0.5 * rho * ke;
  W[3 + ndim] = a1;
}

// Physical flux F^d (alpha component zero) of a state with known thermo
// (Section 3.2).
static void phys_flux(int ndim, int d, const real *W, const Thermo &t, real *F) {
  int E = 2 + ndim, A = 3 + ndim;
  real u = t.vel[d];
  F[0] = W[0] * u;
  F[1] = W[1] * u;
  for (int j = 0; j < ndim; ++j) F[2 + j] = W[2 + j] * u;
  F[2 + d] = F[2 + d] + t.p;
  F[E] = (W[E] + t.p) * u;
  F[A] = 0.0;
}

// Everything the scheme needs at one node, computed once per node and
// direction (steps 1 and 7 of the WCNS algorithm, Section 4.2).
struct Node {
  real W[7];   // conservative state
  real V[7];   // primitive state
  Thermo t;    // mixture thermodynamics
  real F[7];   // physical flux F^d (alpha component zero)
  real G[7];   // G^d = F^d + (0, ..., alpha1 u_d)
  real un;     // normal velocity u_d
};

static void node_prep(const Eos &e, int ndim, int d, const real *W, Node &nd) {
  const int nf = ndim + 4;
  for (int q = 0; q < nf; ++q) nd.W[q] = W[q];
  OC_ROW(ROW_NODE_EOS);
  nd.t = thermo(e, ndim, W);
  nd.V[0] = W[0];
  nd.V[1] = W[1];
  for (int j = 0; j < ndim; ++j) nd.V[2 + j] = nd.t.vel[j];
  nd.V[2 + ndim] = nd.t.p;
  nd.V[3 + ndim] = W[3 + ndim];
  OC_ROW(ROW_NODE_FLUX);
  phys_flux(ndim, d, W, nd.t, nd.F);
  nd.un = nd.t.vel[d];
  for (int q = 0; q < nf; ++q) nd.G[q] = nd.F[q];
  nd.G[3 + ndim] = W[3 + ndim] * nd.un;
}

// ---------------------------------------------------------------------------
// Section 3.1-3.2: HLLC flux G^HLLC(W_L, W_R) in direction d, and u* = s*.
// ---------------------------------------------------------------------------
static real sign_of(real x) {
  if (x > 0.0) return 1.0;
  if (x < 0.0) return -1.0;
  return 0.0;
}

static void hllc_flux(int ndim, int d, const real *WL, const Thermo &tL, const real *FL,
                      const real *WR, const Thermo &tR, const real *FR, real *G, real *ustar) {
  const int nf = ndim + 4;
  const int E = 2 + ndim, A = 3 + ndim;
  real uL = tL.vel[d], uR = tR.vel[d];
  // Einfeldt wave speeds with arithmetic averages.
  real ubar = 0.5 * (uL + uR);
  real cbar = 0.5 * (tL.c + tR.c);
  real sL = o_min(ubar - cbar, uL - tL.c);
  real sR = o_max(ubar + cbar, uR + tR.c);
  // Batten contact speed.
  real num = tR.p - tL.p + tL.rho * uL * (sL - uL) - tR.rho * uR * (sR - uR);
  real den = tL.rho * (sL - uL) - tR.rho * (sR - uR);
  real ss = num / den;
  // Star states W*_L, W*_R.
  real WsL[7], WsR[7];
  {
    real chi = (sL - uL) / (sL - ss);
    WsL[0] = chi * WL[0];
    WsL[1] = chi * WL[1];
    for (int j = 0; j < ndim; ++j) WsL[2 + j] = chi * (tL.rho * tL.vel[j]);
    WsL[2 + d] = chi * (tL.rho * ss);
    WsL[E] = chi * (WL[E] + (ss - uL) * (tL.rho * ss + tL.p / (sL - uL)));
    WsL[A] = WL[A];
  }
  {
    real chi = (sR - uR) / (sR - ss);
    WsR[0] = chi * WR[0];
    WsR[1] = chi * WR[1];
    for (int j = 0; j < ndim; ++j) WsR[2 + j] = chi * (tR.rho * tR.vel[j]);
    WsR[2 + d] = chi * (tR.rho * ss);
    WsR[E] = chi * (WR[E] + (ss - uR) * (tR.rho * ss + tR.p / (sR - uR)));
    WsR[A] = WR[A];
  }
  real sm = o_min(0.0, sL);
  real sp = o_max(0.0, sR);
  real sg = sign_of(ss);
  real wl = 0.5 * (1.0 + sg);
  real wr = 0.5 * (1.0 - sg);
  for (int q = 0; q < nf - 1; ++q) {
    G[q] = wl * (FL[q] + sm * (WsL[q] - WL[q])) + wr * (FR[q] + sp * (WsR[q] - WR[q]));
  }
  // alpha flux, upwinded by the contact speed; u_hat = s*.
  G[A] = wl * (WL[A] * ss) + wr * (WR[A] * ss);
  *ustar = ss;
}

// ---------------------------------------------------------------------------
// Appendix A: characteristic projection in direction d at a midpoint, built
// from arithmetic means of a1r1, a2r2, rho and c at the two adjacent nodes.
// Characteristic ordering: 0 = (u_n - c) wave, 1..2 = partial densities,
// 3.. = tangential velocities, nf-2 = alpha1, nf-1 = (u_n + c) wave.
// ---------------------------------------------------------------------------
static void char_matrices(int ndim, int d, const real *Wa, const Thermo &ta, const real *Wb,
                          const Thermo &tb, real *R, real *Rinv) {
  const int nf = ndim + 4;
  const int P = 2 + ndim, A = 3 + ndim, n = 2 + d;
  real ar1 = 0.5 * (Wa[0] + Wb[0]);
  real ar2 = 0.5 * (Wa[1] + Wb[1]);
  real rho = ar1 + ar2;
  real c = 0.5 * (ta.c + tb.c);
  for (int q = 0; q < nf * nf; ++q) {
    R[q] = 0.0;
    Rinv[q] = 0.0;
  }
  // Rinv: U = Rinv V
  Rinv[0 * nf + n] = 1.0;
  Rinv[0 * nf + P] = -1.0 / (rho * c);
  Rinv[1 * nf + 0] = 1.0;
  Rinv[1 * nf + P] = -ar1 / (rho * c * c);
  Rinv[2 * nf + 1] = 1.0;
  Rinv[2 * nf + P] = -ar2 / (rho * c * c);
  int row = 3;
  for (int j = 0; j < ndim; ++j) {
    if (j == d) continue;
    Rinv[row * nf + 2 + j] = 1.0;
    ++row;
  }
  Rinv[(nf - 2) * nf + A] = 1.0;
  Rinv[(nf - 1) * nf + n] = 1.0;
  Rinv[(nf - 1) * nf + P] = 1.0 / (rho * c);
  // R: V = R U
  R[0 * nf + 0] = -ar1 / (2.0 * c);
  R[0 * nf + 1] = 1.0;
  R[0 * nf + (nf - 1)] = ar1 / (2.0 * c);
  R[1 * nf + 0] = -ar2 / (2.0 * c);
  R[1 * nf + 2] = 1.0;
  R[1 * nf + (nf - 1)] = ar2 / (2.0 * c);
  R[n * nf + 0] = 0.5;
  R[n * nf + (nf - 1)] = 0.5;
  row = 3;
  for (int j = 0; j < ndim; ++j) {
    if (j == d) continue;
    R[(2 + j) * nf + row] = 1.0;
    ++row;
  }
  R[P * nf + 0] = -rho * c / 2.0;
  R[P * nf + (nf - 1)] = rho * c / 2.0;
  R[A * nf + (nf - 2)] = 1.0;
}

// y = M x.  Structural zeros of M are skipped and unit entries add x
// directly; for finite data this is bit-identical to the dense product and
// makes the op-counting build count only the work a sparse product does.
static void matvec(int nf, const real *M, const real *x, real *y) {
  for (int r = 0; r < nf; ++r) {
    real s = 0.0;
    bool first = true;
    for (int q = 0; q < nf; ++q) {
      real m = M[r * nf + q];
      if (m == 0.0) continue;
      real term = (m == 1.0) ? x[q] : m * x[q];
      s = first ? term : s + term;
      first = false;
    }
    y[r] = s;
  }
}

// ---------------------------------------------------------------------------
// Section 4.3: incremental-stencil WENO interpolation, left-biased, to the
// midpoint i+1/2 from u[0..4] = u_{i-2} .. u_{i+2}.
// ---------------------------------------------------------------------------
struct IsOut {
  real value;
  real omega[4];
  real beta[5];  // beta0, beta1, beta01, beta2, beta3
  real tau5;
};

static IsOut wcnsis_left(const real *u, double eps) {
  const real &um2 = u[0], &um1 = u[1], &u0 = u[2], &up1 = u[3], &up2 = u[4];
  IsOut o;
  // Sub-stencil interpolants S0..S3.
  real s[4];
  s[0] = 0.5 * (u0 + up1);
  s[1] = 0.5 * (-um1 + 3.0 * u0);
  s[2] = 0.125 * (3.0 * u0 + 6.0 * up1 - up2);  // x/8 == x*0.125 exactly
  s[3] = 0.125 * (3.0 * um2 - 10.0 * um1 + 15.0 * u0);
  // Smoothness indicators.
  real b0 = (u0 - up1) * (u0 - up1);
  real b1 = (um1 - u0) * (um1 - u0);
  real t01a = um1 - 2.0 * u0 + up1, t01b = um1 - up1;
  real b01 = (13.0 / 12.0) * t01a * t01a + 0.25 * t01b * t01b;
  real t2a = u0 - 2.0 * up1 + up2, t2b = 3.0 * u0 - 4.0 * up1 + up2;
  real b2 = (13.0 / 12.0) * t2a * t2a + 0.25 * t2b * t2b;
  real t3a = um2 - 2.0 * um1 + u0, t3b = um2 - 4.0 * um1 + 3.0 * u0;
  real b3 = (13.0 / 12.0) * t3a * t3a + 0.25 * t3b * t3b;
  // Reference smoothness indicator tau5.
  real t5a = up2 - 4.0 * up1 + 6.0 * u0 - 4.0 * um1 + um2;
  real t5b = up2 - 2.0 * up1 + 2.0 * um1 - um2;
  real tau5 = (13.0 / 12.0) * t5a * t5a + 0.25 * t5b * t5b;
  // Nonlinear weights.
  const double d[4] = {15.0 / 32.0, 5.0 / 32.0, 5.0 / 16.0, 1.0 / 16.0};
  real beta[4] = {b0, b1, b2, b3};
  real eta[4];
  real r01 = tau5 / (b01 + eps);
  for (int k = 0; k < 4; ++k) {
    real rk = tau5 / (beta[k] + eps);
    if (k < 2)
      eta[k] = d[k] * (1.0 + rk * r01);
    else
      eta[k] = d[k] * (1.0 + rk);
  }
  real sum = eta[0] + eta[1] + eta[2] + eta[3];
  real val = 0.0;
  for (int k = 0; k < 4; ++k) {
    o.omega[k] = eta[k] / sum;
    val = val + o.omega[k] * s[k];
  }
  o.value = val;
  o.beta[0] = b0;
  o.beta[1] = b1;
  o.beta[2] = b01;
  o.beta[3] = b2;
  o.beta[4] = b3;
  o.tau5 = tau5;
  return o;
}

// ---------------------------------------------------------------------------
// Section 4.1: HCS reconstructed flux at i+1/2 from the midpoint value gt and
// node values g[0..5] = g_{i-2} .. g_{i+3} (eq. for G-hat, psi = 256/175).
// ---------------------------------------------------------------------------
static const double HCS_PSI = 256.0 / 175.0;

static real hcs_recon(real gt, const real *g) {
  const double psi = HCS_PSI;
  const double c1 = 75.0 * psi / 128.0 - 37.0 / 60.0;
  const double c2 = 25.0 * psi / 256.0 - 2.0 / 15.0;
  const double c3 = 3.0 * psi / 256.0 - 1.0 / 60.0;
  return psi * gt - c1 * (g[2] + g[3]) + c2 * (g[1] + g[4]) - c3 * (g[0] + g[5]);
}

// ---------------------------------------------------------------------------
// Section 5: limiter helpers.
// ---------------------------------------------------------------------------
// theta solving (1-theta) fA + theta fB = eps, with the paper's three cases.
static real limiter_theta(real fA, real fB, double eps) {
  if (fA < eps) return 0.0;
  if (fB < eps) return (fA - eps) / (fA - fB);
  return 1.0;
}

static real alpha_k(int ndim, const real *W, int k) {
  return k == 1 ? W[3 + ndim] : 1.0 - W[3 + ndim];
}

// Section 5.1, Algorithms 1-3 and the hard switch, for one interpolated
// state Wt limited toward the node state Wn.  Returns 1 if any theta < 1,
// sets *hard if the hard switch fired.
static int interp_limit(const Eos &e, const oc_config &cfg, int ndim, const real *Wn, real *Wt,
                        int *hard) {
  const int nf = ndim + 4;
  int limited = 0;
  // Algorithm 1: partial densities, k = 1 then 2.
  for (int k = 1; k <= 2; ++k) {
    real th = limiter_theta(Wn[k - 1], Wt[k - 1], cfg.eps_ar);
    if (th < 1.0) {
      limited = 1;
      for (int q = 0; q < nf; ++q) Wt[q] = (1.0 - th) * Wn[q] + th * Wt[q];
    }
  }
  // Algorithm 2: volume fractions, k = 1 then 2.
  for (int k = 1; k <= 2; ++k) {
    real th = limiter_theta(alpha_k(ndim, Wn, k), alpha_k(ndim, Wt, k), cfg.eps_a);
    if (th < 1.0) {
      limited = 1;
      for (int q = 0; q < nf; ++q) Wt[q] = (1.0 - th) * Wn[q] + th * Wt[q];
    }
  }
  // Algorithm 3: rho*ctilde^2.
  {
    real th = limiter_theta(rho_ct2_of(e, ndim, Wn), rho_ct2_of(e, ndim, Wt), cfg.eps_rc);
    if (th < 1.0) {
      limited = 1;
      for (int q = 0; q < nf; ++q) Wt[q] = (1.0 - th) * Wn[q] + th * Wt[q];
    }
  }
  // Hard switch.
  *hard = 0;
  if (Wt[0] < cfg.hs_ar || Wt[1] < cfg.hs_ar || alpha_k(ndim, Wt, 1) < cfg.hs_a ||
      alpha_k(ndim, Wt, 2) < cfg.hs_a || rho_ct2_of(e, ndim, Wt) < cfg.hs_rc) {
    *hard = 1;
    for (int q = 0; q < nf; ++q) Wt[q] = Wn[q];
  }
  return limited;
}

// Euler half states of Section 5.2:
//   W_i^{+}     = W_i     - 2 lam (G^-_{i+1/2} - F_i)
//   W_{i+1}^{-} = W_{i+1} + 2 lam (G^+_{i+1/2} - F_{i+1})
static void half_plus(int nf, const real *Wi, const real *Fi, const real *Gm, real lam, real *out) {
  for (int q = 0; q < nf; ++q) out[q] = Wi[q] - 2.0 * lam * (Gm[q] - Fi[q]);
}
static void half_minus(int nf, const real *Wi1, const real *Fi1, const real *Gp, real lam,
                       real *out) {
  for (int q = 0; q < nf; ++q) out[q] = Wi1[q] + 2.0 * lam * (Gp[q] - Fi1[q]);
}

enum { F_AR1, F_AR2, F_A1, F_A2, F_RCT2 };
static real limited_quantity(const Eos &e, int ndim, const real *W, int which) {
  switch (which) {
    case F_AR1: return W[0];
    case F_AR2: return W[1];
    case F_A1: return alpha_k(ndim, W, 1);
    case F_A2: return alpha_k(ndim, W, 2);
    default: return rho_ct2_of(e, ndim, W);
  }
}

// Section 5.2, Algorithms 4-6 and the flux hard switch at one midpoint.
// Gm/Gp hold the high-order fluxes G^-_{i+1/2}, G^+_{i+1/2} on entry and the
// limited fluxes on exit.  Returns 1 if any theta < 1.
static int flux_limit(const Eos &e, const oc_config &cfg, int ndim, const real *Wi,
                      const real *Wi1, const real *Fi, const real *Fi1, const real *GHm,
                      const real *GHp, real lam, real *Gm, real *Gp, int *hard) {
  const int nf = ndim + 4;
  int limited = 0;
  real Ap[7], Am[7], Bp[7], Bm[7];
  half_plus(nf, Wi, Fi, GHm, lam, Ap);     // W_i^{HLLC,+}
  half_minus(nf, Wi1, Fi1, GHp, lam, Am);  // W_{i+1}^{HLLC,-}
  half_plus(nf, Wi, Fi, Gm, lam, Bp);      // W_i^{+} from the current G^-
  half_minus(nf, Wi1, Fi1, Gp, lam, Bm);   // W_{i+1}^{-} from the current G^+
  // Algorithm 4 (k = 1, 2), Algorithm 5 (k = 1, 2), Algorithm 6.
  const int order[5] = {F_AR1, F_AR2, F_A1, F_A2, F_RCT2};
  for (int s = 0; s < 5; ++s) {
    int which = order[s];
    double eps = (which == F_AR1 || which == F_AR2) ? cfg.eps_ar
                 : (which == F_A1 || which == F_A2) ? cfg.eps_a
                                                    : cfg.eps_rc;
    real thp = limiter_theta(limited_quantity(e, ndim, Ap, which),
                             limited_quantity(e, ndim, Bp, which), eps);
    real thm = limiter_theta(limited_quantity(e, ndim, Am, which),
                             limited_quantity(e, ndim, Bm, which), eps);
    real th = o_min(thp, thm);
    if (th < 1.0) {
      limited = 1;
      for (int q = 0; q < nf; ++q) {
        Gp[q] = (1.0 - th) * GHp[q] + th * Gp[q];
        Gm[q] = (1.0 - th) * GHm[q] + th * Gm[q];
      }
      // The half states follow the blended fluxes.
      half_plus(nf, Wi, Fi, Gm, lam, Bp);
      half_minus(nf, Wi1, Fi1, Gp, lam, Bm);
    }
  }
  // Hard switch on W_i^{***,+} and W_{i+1}^{***,-}.
  *hard = 0;
  const real *B[2] = {Bp, Bm};
  for (int s = 0; s < 2; ++s) {
    const real *X = B[s];
    if (X[0] < cfg.hs_ar || X[1] < cfg.hs_ar || alpha_k(ndim, X, 1) < cfg.hs_a ||
        alpha_k(ndim, X, 2) < cfg.hs_a || rho_ct2_of(e, ndim, X) < cfg.hs_rc)
      *hard = 1;
  }
  if (*hard) {
    for (int q = 0; q < nf; ++q) {
      Gp[q] = GHp[q];
      Gm[q] = GHm[q];
    }
  }
  return limited;
}

// ---------------------------------------------------------------------------
// Section 4.2: the nine-step WCNS midpoint algorithm, followed by the first-
// order HLLC fluxes (Section 3.2) and the flux limiter (Section 5.2).
// nodes[j] is node i-2+j, j = 0..5; the midpoint is i+1/2.
// ---------------------------------------------------------------------------
static void midpoint_flux(const Eos &e, const oc_config &cfg, int ndim, int d, const Node *const *nodes,
                          real lam, real *Gm, real *Gp, oc_stats *st) {
  const int nf = ndim + 4;
  const int A = 3 + ndim;
  const Node &ni = *nodes[2];
  const Node &ni1 = *nodes[3];
  st->midpoints++;

  // First-order HLLC flux from (W_i, W_{i+1}) and its split (Section 3.2).
  OC_ROW(ROW_HLLC1);
  real GH[7], uH;
  hllc_flux(ndim, d, ni.W, ni.t, ni.F, ni1.W, ni1.t, ni1.F, GH, &uH);
  real GHm[7], GHp[7];
  for (int q = 0; q < nf; ++q) {
    GHm[q] = GH[q];
    GHp[q] = GH[q];
  }
  GHm[A] = GH[A] - ni.W[A] * uH;
  GHp[A] = GH[A] - ni1.W[A] * uH;
  if (cfg.scheme == OC_SCHEME_HLLC1) {
    for (int q = 0; q < nf; ++q) {
      Gm[q] = GHm[q];
      Gp[q] = GHp[q];
    }
    return;
  }

  // Step 1 (W -> V) is done per node in node_prep.
  // Step 2: project the six nodes with Rinv_{i+1/2}.
  OC_ROW(ROW_PROJECT);
  real R[49], Rinv[49];
  char_matrices(ndim, d, ni.W, ni.t, ni1.W, ni1.t, R, Rinv);
  real U[6][7];
  for (int j = 0; j < 6; ++j) matvec(nf, Rinv, nodes[j]->V, U[j]);
  // Step 3: left- and right-biased IS interpolation of every characteristic
  // variable.  The right-biased one is the left-biased formula applied to
  // the stencil mirrored about i+1/2.
  OC_ROW(ROW_WCNS_IS);
  real UL[7], UR[7];
  for (int q = 0; q < nf; ++q) {
    real sl[5] = {U[0][q], U[1][q], U[2][q], U[3][q], U[4][q]};
    real sr[5] = {U[5][q], U[4][q], U[3][q], U[2][q], U[1][q]};
    UL[q] = wcnsis_left(sl, cfg.eps_is).value;
    UR[q] = wcnsis_left(sr, cfg.eps_is).value;
  }
  // Step 4: back-project.
  OC_ROW(ROW_BACKPROJECT);
  real VL[7], VR[7];
  matvec(nf, R, UL, VL);
  matvec(nf, R, UR, VR);
  // Step 5: V -> W.
  real WL[7], WR[7];
  prim_to_cons(e, ndim, VL, WL);
  prim_to_cons(e, ndim, VR, WR);
  // Interpolation limiter (Section 5.1): left toward W_i, right toward W_{i+1}.
  OC_ROW(ROW_INTERP_LIMIT);
  if (cfg.scheme == OC_SCHEME_PP_WCNS_IS) {
    int hard = 0;
    st->interp_limited += interp_limit(e, cfg, ndim, ni.W, WL, &hard);
    st->interp_hard += hard;
    st->interp_limited += interp_limit(e, cfg, ndim, ni1.W, WR, &hard);
    st->interp_hard += hard;
  }
  // Step 6: midpoint HLLC flux and velocity.
  OC_ROW(ROW_MID_HLLC);
  Thermo tL = thermo(e, ndim, WL);
  Thermo tR = thermo(e, ndim, WR);
  real FL[7], FR[7];
  phys_flux(ndim, d, WL, tL, FL);
  phys_flux(ndim, d, WR, tR, FR);
  real Gt[7], ut;
  hllc_flux(ndim, d, WL, tL, FL, WR, tR, FR, Gt, &ut);
  // Step 7 (node fluxes G_j, velocities u_j) is done per node in node_prep.
  // Step 8: HCS reconstruction of G-hat and u-hat.
  OC_ROW(ROW_HCS);
  real Gh[7];
  for (int q = 0; q < nf; ++q) {
    real g[6];
    for (int j = 0; j < 6; ++j) g[j] = nodes[j]->G[q];
    Gh[q] = hcs_recon(Gt[q], g);
  }
  real un[6];
  for (int j = 0; j < 6; ++j) un[j] = nodes[j]->un;
  real uh = hcs_recon(ut, un);
  // Step 9: the non-conservative split G^-_{i+1/2}, G^+_{i+1/2}.
  for (int q = 0; q < nf; ++q) {
    Gm[q] = Gh[q];
    Gp[q] = Gh[q];
  }
  Gm[A] = Gh[A] - ni.W[A] * uh;
  Gp[A] = Gh[A] - ni1.W[A] * uh;

  // Flux limiter (Section 5.2).
  OC_ROW(ROW_FLUX_LIMIT);
  if (cfg.scheme == OC_SCHEME_PP_WCNS_IS) {
    int hard = 0;
    st->flux_limited +=
        flux_limit(e, cfg, ndim, ni.W, ni1.W, ni.F, ni1.F, GHm, GHp, lam, Gm, Gp, &hard);
    st->flux_hard += hard;
  }
}

// ---------------------------------------------------------------------------
// Grid helpers.
// ---------------------------------------------------------------------------
static Eos make_eos(const oc_config &c) {
  Eos e;
  e.g1 = c.gamma_l;
  e.p1 = c.pinf_l;
  e.g2 = c.gamma_g;
  e.p2 = 0.0;
  e.r1 = 1.0 / (e.g1 - 1.0);
  e.r2 = 1.0 / (e.g2 - 1.0);
  e.q1 = e.g1 * e.p1 / (e.g1 - 1.0);
  e.q2 = e.g2 * e.p2 / (e.g2 - 1.0);
  return e;
}

static long ncells(const oc_config &c) {
  long n = 1;
  for (int d = 0; d < c.ndim; ++d) n *= c.n[d];
  return n;
}

static double spacing(const oc_config &c, int d) { return (c.hi[d] - c.lo[d]) / c.n[d]; }

// SoA layout [nf][n_z][n_y][n_x]: x is the fastest index.
static long cell_index(const oc_config &c, const int *ijk) {
  long idx = 0;
  for (int d = c.ndim - 1; d >= 0; --d) idx = idx * c.n[d] + ijk[d];
  return idx;
}

// Fill one line of conservative states along direction d, including three
// ghost layers per side, from the interior cells of the SoA array W.
static void gather_line(const oc_config &c, const double *W, int d, int *ijk,
                        std::vector<real> &line) {
  const int nf = c.ndim + 4;
  const int n = c.n[d];
  const long N = ncells(c);
  line.assign((size_t)(n + 6) * nf, 0.0);
  for (int g = 0; g < n + 6; ++g) {
    int i = g - 3;
    real *dst = &line[(size_t)g * nf];
    int side = i < 0 ? 0 : 1;
    int kind = (i < 0 || i >= n) ? c.bc[d][side] : -1;
    int src = i;
    bool flip = false;
    if (kind == OC_BC_TRANSMISSIVE) {
      src = i < 0 ? 0 : n - 1;
    } else if (kind == OC_BC_PERIODIC) {
      src = ((i % n) + n) % n;
    } else if (kind == OC_BC_SYMMETRY) {
      src = i < 0 ? -1 - i : 2 * n - 1 - i;
      flip = true;
    } else if (kind == OC_BC_DIRICHLET) {
      const double *face = c.dir_face[d][side];
      if (face) {
        // position of this line on the face: the other axes, lower fastest
        long fidx = 0, mult = 1;
        for (int dd = 0; dd < c.ndim; ++dd) {
          if (dd == d) continue;
          fidx += mult * ijk[dd];
          mult *= c.n[dd];
        }
        const long nface = mult;
        for (int q = 0; q < nf; ++q) dst[q] = face[(size_t)q * nface + fidx];
      } else {
        for (int q = 0; q < nf; ++q) dst[q] = c.dirichlet[d][side][q];
      }
      continue;
    }
    int save = ijk[d];
    ijk[d] = src;
    long idx = cell_index(c, ijk);
    ijk[d] = save;
    for (int q = 0; q < nf; ++q) dst[q] = W[(size_t)q * N + idx];
    if (flip) dst[2 + d] = -dst[2 + d];
  }
}

// (|u_d| + c)_max over the interior cells, per direction (Section 3.3).
static void max_wavespeed_impl(const oc_config &c, const double *W, double *out) {
  const int nf = c.ndim + 4;
  const long N = ncells(c);
  Eos e = make_eos(c);
  for (int d = 0; d < 3; ++d) out[d] = 0.0;
  real w[7] = {};
  auto take = [&](const real *ws) {
    Thermo t = thermo(e, c.ndim, ws);
    for (int d = 0; d < c.ndim; ++d) {
      double s = o_val(o_abs(t.vel[d]) + t.c);
      if (!(s <= out[d])) out[d] = s;  // a NaN wins and stays
    }
  };
  for (long idx = 0; idx < N; ++idx) {
    for (int q = 0; q < nf; ++q) w[q] = W[(size_t)q * N + idx];
    take(w);
  }
  // Dirichlet ghost states enter the boundary midpoints' fluxes like cells,
  // so their wave speeds bound dt as well (the other kinds of ghost copy
  // interior cells and add nothing).
  for (int dd = 0; dd < c.ndim; ++dd) {
    for (int side = 0; side < 2; ++side) {
      if (c.bc[dd][side] != OC_BC_DIRICHLET) continue;
      const double *face = c.dir_face[dd][side];
      const long nface = face ? N / c.n[dd] : 1;
      for (long k = 0; k < nface; ++k) {
        for (int q = 0; q < nf; ++q) w[q] = face ? face[(size_t)q * nface + k] : c.dirichlet[dd][side][q];
        take(w);
      }
    }
  }
}

static void rhs_impl(const oc_config &c, const double *W, double *dWdt, double dt, oc_stats *st,
                     const double *smax_given = nullptr) {
  const int nf = c.ndim + 4;
  const long N = ncells(c);
  Eos e = make_eos(c);
  for (long q = 0; q < (long)nf * N; ++q) dWdt[q] = 0.0;
  // Directional split (Section 3.3): sigma_d = tau_d / sum(tau), with
  // tau_d = (|u_d| + c)_max / dx_d, and lambda_d = dt / (dx_d sigma_d).
  double smax[3];
  if (smax_given) {
    for (int d = 0; d < 3; ++d) smax[d] = smax_given[d];
  } else {
    OC_ROW(ROW_WAVESPEED);
    max_wavespeed_impl(c, W, smax);
  }
  double tau[3], tsum = 0.0;
  for (int d = 0; d < c.ndim; ++d) {
    tau[d] = smax[d] / spacing(c, d);
    tsum += tau[d];
  }
  std::vector<real> line, Gm, Gp;
  std::vector<Node> nodes;
  for (int d = 0; d < c.ndim; ++d) {
    const int n = c.n[d];
    const double dx = spacing(c, d);
    const double sigma = c.ndim == 1 ? 1.0 : tau[d] / tsum;
    const real lam = dt / (dx * sigma);
    int ijk[3] = {0, 0, 0};
    int other[2], no = 0;
    for (int dd = 0; dd < c.ndim; ++dd)
      if (dd != d) other[no++] = dd;
    long nlines = N / n;
    for (long l = 0; l < nlines; ++l) {
      long rem = l;
      for (int o = 0; o < no; ++o) {
        ijk[other[o]] = (int)(rem % c.n[other[o]]);
        rem /= c.n[other[o]];
      }
      ijk[d] = 0;
      gather_line(c, W, d, ijk, line);
      nodes.assign(n + 6, Node());
      for (int g = 0; g < n + 6; ++g) node_prep(e, c.ndim, d, &line[(size_t)g * nf], nodes[g]);
      // Midpoint m sits between line nodes m+2 and m+3 (cells m-1 and m),
      // m = 0 .. n.
      Gm.assign((size_t)(n + 1) * nf, 0.0);
      Gp.assign((size_t)(n + 1) * nf, 0.0);
      for (int m = 0; m <= n; ++m) {
        const Node *np[6];
        for (int j = 0; j < 6; ++j) np[j] = &nodes[m + j];
        midpoint_flux(e, c, c.ndim, d, np, lam, &Gm[(size_t)m * nf], &Gp[(size_t)m * nf], st);
      }
      // Semi-discrete update: dW_i/dt -= (G^-_{i+1/2} - G^+_{i-1/2}) / dx.
      OC_ROW(ROW_UPDATE);
      for (int i = 0; i < n; ++i) {
        ijk[d] = i;
        long idx = cell_index(c, ijk);
        for (int q = 0; q < nf; ++q) {
          real upd = (Gm[(size_t)(i + 1) * nf + q] - Gp[(size_t)i * nf + q]) / dx;
          dWdt[(size_t)q * N + idx] = o_val(dWdt[(size_t)q * N + idx] - upd);
        }
      }
    }
  }
}

// Shu-Osher SSPRK3 (Section 5.3 cites it; standard three-stage form):
//   W1 = W + dt L(W);  W2 = 3/4 W + 1/4 (W1 + dt L(W1));
//   W^{n+1} = 1/3 W + 2/3 (W2 + dt L(W2)).
static void rk3_impl(const oc_config &c, double *W, double dt, oc_stats *st) {
  const int nf = c.ndim + 4;
  const long N = ncells(c);
  const size_t M = (size_t)nf * N;
  std::vector<double> W0(W, W + M), W1(M), W2(M), L(M);
  // the stage combinations in `real` arithmetic (the op-counting build
  // books them to their own step; the values are the same doubles)
  const real h = dt;
  rhs_impl(c, W0.data(), L.data(), dt, st);
  OC_ROW(ROW_COMBINE);
  for (size_t q = 0; q < M; ++q) W1[q] = o_val(real(W0[q]) + h * real(L[q]));
  rhs_impl(c, W1.data(), L.data(), dt, st);
  OC_ROW(ROW_COMBINE);
  for (size_t q = 0; q < M; ++q)
    W2[q] = o_val(real(0.75) * real(W0[q]) + real(0.25) * (real(W1[q]) + h * real(L[q])));
  rhs_impl(c, W2.data(), L.data(), dt, st);
  OC_ROW(ROW_COMBINE);
  for (size_t q = 0; q < M; ++q)
    W[q] = o_val(real(1.0 / 3.0) * real(W0[q]) + real(2.0 / 3.0) * (real(W2[q]) + h * real(L[q])));
  OC_ROW(ROW_OTHER);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI of the oracle (loaded by the tests through ctypes).
// ---------------------------------------------------------------------------
extern "C" {

int oc_nfields(const oc_config *c) { return c->ndim + 4; }

void oc_rhs(const oc_config *c, const double *W, double *dWdt, double dt, oc_stats *st) {
  rhs_impl(*c, W, dWdt, dt, st);
}

// As oc_rhs, with the maxima of (|u_d| + c) that set sigma_d supplied by the
// caller (used to evaluate the RHS of a sub-box of a larger grid).
void oc_rhs_smax(const oc_config *c, const double *W, double *dWdt, double dt, const double *smax3,
                 oc_stats *st) {
  rhs_impl(*c, W, dWdt, dt, st, smax3);
}

void oc_max_wavespeed(const oc_config *c, const double *W, double *out3) {
  max_wavespeed_impl(*c, W, out3);
}

void oc_rk3_step(const oc_config *c, double *W, double dt, oc_stats *st) { rk3_impl(*c, W, dt, st); }

// Advance from t0 to t_end.  With dt_fixed > 0 every step uses dt_fixed
// (the last one clipped to land on t_end); otherwise dt = cfl / sum_d tau_d
// from the state at the start of the step (Section 3.3).  max_steps bounds
// the loop.
int oc_advance_to(const oc_config *c, double *W, double t0, double t_end, double cfl,
                  double dt_fixed, long max_steps, double *t_out, long *steps_out, oc_stats *st) {
  double t = t0;
  long steps = 0;
  while (t < t_end && steps < max_steps) {
    double dt;
    if (dt_fixed > 0.0) {
      dt = dt_fixed;
    } else {
      double smax[3];
      max_wavespeed_impl(*c, W, smax);
      double tsum = 0.0;
      for (int d = 0; d < c->ndim; ++d) tsum += smax[d] / spacing(*c, d);
      dt = cfl / tsum;
    }
    bool last = t + dt >= t_end;
    if (last) dt = t_end - t;
    rk3_impl(*c, W, dt, st);
    t = last ? t_end : t + dt;
    ++steps;
  }
  *t_out = t;
  *steps_out = steps;
  return 0;
}

// --- unit-level entry points used by the pin tests -------------------------

// Outputs (p, rho*c^2, rho*ctilde^2, gamma_bar, pinf_bar, c).
void oc_thermo(const oc_config *c, const double *W, double *out6) {
  Eos e = make_eos(*c);
  real w[7] = {};
  for (int q = 0; q < c->ndim + 4; ++q) w[q] = W[q];
  Thermo t = thermo(e, c->ndim, w);
  out6[0] = o_val(t.p);
  out6[1] = o_val(t.rho_c2);
  out6[2] = o_val(t.rho_ct2);
  out6[3] = o_val(mix_gamma(e, w[3 + c->ndim]));
  out6[4] = o_val(mix_pinf(e, w[3 + c->ndim]));
  out6[5] = o_val(t.c);
}

void oc_prim_to_cons(const oc_config *c, const double *V, double *W) {
  Eos e = make_eos(*c);
  real v[7] = {}, w[7] = {};
  for (int q = 0; q < c->ndim + 4; ++q) v[q] = V[q];
  prim_to_cons(e, c->ndim, v, w);
  for (int q = 0; q < c->ndim + 4; ++q) W[q] = o_val(w[q]);
}

void oc_cons_to_prim(const oc_config *c, const double *W, double *V) {
  Eos e = make_eos(*c);
  real v[7] = {}, w[7] = {};
  for (int q = 0; q < c->ndim + 4; ++q) w[q] = W[q];
  cons_to_prim(e, c->ndim, w, v);
  for (int q = 0; q < c->ndim + 4; ++q) V[q] = o_val(v[q]);
}

// G^d(W) = F^d(W) + (0, ..., alpha1 u_d).
void oc_phys_flux(const oc_config *c, int d, const double *W, double *G) {
  Eos e = make_eos(*c);
  const int nf = c->ndim + 4;
  real w[7] = {};
  for (int q = 0; q < nf; ++q) w[q] = W[q];
  Node nd;
  node_prep(e, c->ndim, d, w, nd);
  for (int q = 0; q < nf; ++q) G[q] = o_val(nd.G[q]);
}

void oc_hllc(const oc_config *c, int d, const double *WL, const double *WR, double *G,
             double *ustar) {
  Eos e = make_eos(*c);
  const int nf = c->ndim + 4;
  real wl[7] = {}, wr[7] = {}, g[7], us;
  for (int q = 0; q < nf; ++q) {
    wl[q] = WL[q];
    wr[q] = WR[q];
  }
  Node nl, nr;
  node_prep(e, c->ndim, d, wl, nl);
  node_prep(e, c->ndim, d, wr, nr);
  hllc_flux(c->ndim, d, nl.W, nl.t, nl.F, nr.W, nr.t, nr.F, g, &us);
  for (int q = 0; q < nf; ++q) G[q] = o_val(g[q]);
  *ustar = o_val(us);
}

// Outputs the HLLC wave speeds (sL, s*, sR) and the two star states,
// recomputed here from the same formulas as hllc_flux.
void oc_hllc_star(const oc_config *c, int d, const double *WL, const double *WR, double *s3,
                  double *WsL, double *WsR) {
  Eos e = make_eos(*c);
  const int ndim = c->ndim;
  const int E = 2 + ndim, A = 3 + ndim;
  real wl[7] = {}, wr[7] = {};
  for (int q = 0; q < ndim + 4; ++q) {
    wl[q] = WL[q];
    wr[q] = WR[q];
  }
  Thermo tL = thermo(e, ndim, wl), tR = thermo(e, ndim, wr);
  real uL = tL.vel[d], uR = tR.vel[d];
  real ubar = 0.5 * (uL + uR), cbar = 0.5 * (tL.c + tR.c);
  real sL = o_min(ubar - cbar, uL - tL.c);
  real sR = o_max(ubar + cbar, uR + tR.c);
  real ss = (tR.p - tL.p + tL.rho * uL * (sL - uL) - tR.rho * uR * (sR - uR)) /
            (tL.rho * (sL - uL) - tR.rho * (sR - uR));
  s3[0] = o_val(sL);
  s3[1] = o_val(ss);
  s3[2] = o_val(sR);
  const real *Ws[2] = {wl, wr};
  const Thermo *T[2] = {&tL, &tR};
  real sK[2] = {sL, sR};
  double *out[2] = {WsL, WsR};
  for (int s = 0; s < 2; ++s) {
    const real *w = Ws[s];
    const Thermo &t = *T[s];
    real uK = t.vel[d];
    real chi = (sK[s] - uK) / (sK[s] - ss);
    out[s][0] = o_val(chi * w[0]);
    out[s][1] = o_val(chi * w[1]);
    for (int j = 0; j < ndim; ++j) out[s][2 + j] = o_val(chi * (t.rho * t.vel[j]));
    out[s][2 + d] = o_val(chi * (t.rho * ss));
    out[s][E] = o_val(chi * (w[E] + (ss - uK) * (t.rho * ss + t.p / (sK[s] - uK))));
    out[s][A] = o_val(w[A]);
  }
}

void oc_char_matrices(const oc_config *c, int d, const double *Wa, const double *Wb, double *R,
                      double *Rinv) {
  Eos e = make_eos(*c);
  const int nf = c->ndim + 4;
  real wa[7] = {}, wb[7] = {}, r[49], ri[49];
  for (int q = 0; q < nf; ++q) {
    wa[q] = Wa[q];
    wb[q] = Wb[q];
  }
  Thermo ta = thermo(e, c->ndim, wa), tb = thermo(e, c->ndim, wb);
  char_matrices(c->ndim, d, wa, ta, wb, tb, r, ri);
  for (int q = 0; q < nf * nf; ++q) {
    R[q] = o_val(r[q]);
    Rinv[q] = o_val(ri[q]);
  }
}

// out = (value, omega0..3, beta0, beta1, beta01, beta2, beta3, tau5): 11 values.
void oc_wcnsis_left(const double *u5, double eps, double *out11) {
  real u[5];
  for (int j = 0; j < 5; ++j) u[j] = u5[j];
  IsOut o = wcnsis_left(u, eps);
  out11[0] = o_val(o.value);
  for (int k = 0; k < 4; ++k) out11[1 + k] = o_val(o.omega[k]);
  for (int k = 0; k < 5; ++k) out11[5 + k] = o_val(o.beta[k]);
  out11[10] = o_val(o.tau5);
}

double oc_hcs_recon(double gt, const double *g6) {
  real g[6];
  for (int j = 0; j < 6; ++j) g[j] = g6[j];
  return o_val(hcs_recon(gt, g));
}

// One midpoint's limited split fluxes from six node states (nf each, nodes
// i-2 .. i+3 stored consecutively in nodes6).
void oc_midpoint_flux(const oc_config *c, int d, const double *nodes6, double lam, double *Gm,
                      double *Gp, oc_stats *st) {
  Eos e = make_eos(*c);
  const int nf = c->ndim + 4;
  Node nd[6];
  const Node *np[6];
  for (int j = 0; j < 6; ++j) {
    real w[7];
    for (int q = 0; q < nf; ++q) w[q] = nodes6[j * nf + q];
    node_prep(e, c->ndim, d, w, nd[j]);
    np[j] = &nd[j];
  }
  real gm[7], gp[7];
  midpoint_flux(e, *c, c->ndim, d, np, lam, gm, gp, st);
  for (int q = 0; q < nf; ++q) {
    Gm[q] = o_val(gm[q]);
    Gp[q] = o_val(gp[q]);
  }
}

// Limiter entry points for the pin tests (Algorithms 1-3 and 4-6).
int oc_interp_limit(const oc_config *c, const double *Wn, double *Wt, int *hard) {
  Eos e = make_eos(*c);
  const int nf = c->ndim + 4;
  real wn[7] = {}, wt[7] = {};
  for (int q = 0; q < nf; ++q) {
    wn[q] = Wn[q];
    wt[q] = Wt[q];
  }
  int lim = interp_limit(e, *c, c->ndim, wn, wt, hard);
  for (int q = 0; q < nf; ++q) Wt[q] = o_val(wt[q]);
  return lim;
}

int oc_flux_limit(const oc_config *c, int d, const double *Wi, const double *Wi1, const double *GHm,
                  const double *GHp, double lam, double *Gm, double *Gp, int *hard) {
  Eos e = make_eos(*c);
  const int nf = c->ndim + 4;
  real wi[7] = {}, wi1[7] = {}, ghm[7] = {}, ghp[7] = {}, gm[7] = {}, gp[7] = {};
  for (int q = 0; q < nf; ++q) {
    wi[q] = Wi[q];
    wi1[q] = Wi1[q];
    ghm[q] = GHm[q];
    ghp[q] = GHp[q];
    gm[q] = Gm[q];
    gp[q] = Gp[q];
  }
  Node ni, ni1;
  node_prep(e, c->ndim, d, wi, ni);
  node_prep(e, c->ndim, d, wi1, ni1);
  int lim = flux_limit(e, *c, c->ndim, wi, wi1, ni.F, ni1.F, ghm, ghp, lam, gm, gp, hard);
  for (int q = 0; q < nf; ++q) {
    Gm[q] = o_val(gm[q]);
    Gp[q] = o_val(gp[q]);
  }
  return lim;
}

#ifdef ORACLE_COUNT_OPS
void oc_opcount_reset(void) {
  g_oracle_ops = OracleOpCounts{0, 0, 0, 0, 0};
  for (int r = 0; r < ORACLE_NROWS; ++r) g_oracle_rows[r] = OracleOpCounts{0, 0, 0, 0, 0};
  g_oracle_row = ROW_OTHER;
}
// out[5 r + k] = count k (add, mul, div, sqrt, minmax) of step r, r < ORACLE_NROWS
int oc_opcount_rows(unsigned long long *out) {
  for (int r = 0; r < ORACLE_NROWS; ++r) {
    out[5 * r + 0] = g_oracle_rows[r].add;
    out[5 * r + 1] = g_oracle_rows[r].mul;
    out[5 * r + 2] = g_oracle_rows[r].div;
    out[5 * r + 3] = g_oracle_rows[r].sqrt;
    out[5 * r + 4] = g_oracle_rows[r].minmax;
  }
  return ORACLE_NROWS;
}
// out = (add, mul, div, sqrt, minmax)
void oc_opcount_get(unsigned long long *out5) {
  out5[0] = g_oracle_ops.add;
  out5[1] = g_oracle_ops.mul;
  out5[2] = g_oracle_ops.div;
  out5[3] = g_oracle_ops.sqrt;
  out5[4] = g_oracle_ops.minmax;
}
#endif

}  // extern "C"
