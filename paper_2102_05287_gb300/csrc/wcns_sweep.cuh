// Fused directional sweep of the PP-WCNS-IS right-hand side (Wong et al.,
// arXiv 2102.05287) for GB300 (sm_103a).
//
// One launch handles one direction d of one RHS evaluation.  A thread block
// owns a tile of TL lines x TM midpoints along d:
//   1. stage the conservative states of the tile's TM+5 nodes per line
//      (three-cell halo on each side) into shared memory, applying the
//      boundary conditions by index remapping (no ghost arrays in HBM);
//   2. node work, once per node: pressure and sound speed (Sec. 2), the
//      flux G^d including alpha1*u_d (Sec. 3.2);
//   3. one thread per midpoint i+1/2: characteristic projection (App. A),
//      left/right WCNS-IS interpolation (Sec. 4.3), back-projection and
//      V -> W, interpolation limiter (Sec. 5.1, Algs. 1-3), midpoint HLLC
//      (Sec. 3.1-3.2), HCS flux reconstruction (Sec. 4.1), the split
//      G^-/G^+ (Sec. 3.2), first-order HLLC fluxes and the flux limiter
//      (Sec. 5.2, Algs. 4-6);
//   4. cell update dW/dt -= (G^-_{i+1/2} - G^+_{i-1/2})/dx, written to the
//      RHS array or fused with the SSPRK3 stage combine (Sec. 5.3), whose
//      epilogue also reduces max(|u_d| + c) of the new state for the next
//      stage's directional split (Sec. 3.3).
// Consecutive tiles overlap by one midpoint so that every cell's two faces
// are computed inside one block.
//
// Precision: R is the type of the projection, interpolation and HLLC
// arithmetic (double for the FP64 path, float for the mixed path).  Node
// pressure / sound speed, the limiters and all state arithmetic are FP64.
// The interpolation works on deviations from node i: WCNS-IS is exactly
// shift invariant (sub-stencil weights sum to one, smoothness indicators
// use differences), so U~ = U_i + WCNS-IS(U - U_i) and FP32 rounding then
// scales with the local variation instead of the magnitude of the fields.
#pragma once
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "wcns_internal.h"

namespace wcns {

// ---------------------------------------------------------------------------
// Tile shapes: TL lines x TM midpoints, THREADS threads per block.  The
// x sweep takes whole rows of midpoints (coalesced along x); the y/z sweeps
// take a few neighbouring x columns per block.
// ---------------------------------------------------------------------------
template <int TL_, int TM_, int THREADS_>
struct TileT {
  static constexpr int TL = TL_;
  static constexpr int TM = TM_;
  static constexpr int THREADS = THREADS_;
  static constexpr int NS = TM + 5;      // nodes per line
  static constexpr int NN = TL * NS;     // nodes per block
  static constexpr int NM = TL * TM;     // midpoints per block
};
// Tile shapes (lines x midpoints, measured on GB300), 128 threads and two
// blocks per SM except in the 3D x sweep:
// - x in 1D and 2D: 1 x 123 midpoints, 128 nodes, one per thread;
// - y in 2D: 2 x-columns x 64 midpoints, one midpoint per thread (8 % faster
//   than 8 x 59 at 256 threads; the column loads are uncoalesced, but the
//   neighbouring columns' blocks find the sectors in L2);
// - y/z in 3D: 4 x 32 (1 % faster than 8 x 32, 4 % faster than 2 x 64);
// - x in 3D: 2 x 59 (128 nodes; 4 % faster on the 384^3 bubble collapse than
//   3 x 80 at 256 threads, whose 79-cell tiles fit 384-cell rows better,
//   and 3 % faster than 1 x 123).
// Two 128-thread blocks per SM overlap one block's staging and barriers
// with the other's arithmetic.
#ifndef FP64_TM_X
#define FP64_TM_X 123
#endif
template <int NDIM, int DIR>
using Tile = TileT<(DIR == 0) ? (NDIM == 3 ? 2 : 1) : (NDIM == 2 ? 2 : 4),
                   (DIR == 0) ? (NDIM == 3 ? 59 : FP64_TM_X) : (NDIM == 2 ? 64 : 32), 128>;

// Integer tests on FP64 values (no FP64-pipe compare): finite, and
// finite-and-nonnegative (-0 counts as nonnegative, NaN and infinities
// as neither).
__device__ __forceinline__ bool finite64(double v) {
  return (__double2hiint(v) & 0x7FF00000) != 0x7FF00000;
}
__device__ __forceinline__ bool nonneg64(double v) {
  const long long b = __double_as_longlong(v);
  return (b >= 0 && b < 0x7FF0000000000000ll) || b == (long long)0x8000000000000000ull;
}
// x < t for a finite threshold t >= 0, as an integer compare of the bit
// patterns (non-negative doubles order like their bits, negatives are
// below): equal to the FP64 compare for every x that is not a NaN.
__device__ __forceinline__ bool below64(double x, double t) {
  const long long bx = __double_as_longlong(x), bt = __double_as_longlong(t);
  return bx < bt && (bx != (long long)0x8000000000000000ull || bt != 0);
}
// x < 0 and x > 0 for every x that is not a NaN (-0 is neither).
__device__ __forceinline__ bool negative64(double x) {
  const long long b = __double_as_longlong(x);
  return b < 0 && b != (long long)0x8000000000000000ull;
}
__device__ __forceinline__ bool positive64(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7FF0000000000000ll;
}

// a / b in FP64 with five FP64-pipe operations (the FP64 pipe is GB300's
// scarce one; an IEEE division takes about nine): a reciprocal seed y0
// from the approximate FP32 reciprocal of b's leading mantissa bits, b's
// exponent and sign applied with integer operations (|y0 b - 1| < 2^-21);
// one Newton-Raphson step y1 = y0 + y0 (1 - b y0) (relative error below
// 2^-41); the quotient q0 = a y1; and one correction q1 = q0 + y1 (a - b q0)
// with the remainder from a fused multiply-add (Markstein, IBM J. Res.
// Dev. 34 (1990) 111), which leaves q1 within one unit in the last place
// of a / b.  Operands outside the range where that holds (b zero,
// subnormal, not finite or above 2^1021; a not finite or below 2^-959, where
// the remainder would underflow; a / b near the overflow threshold) take the
// IEEE division, except a zero numerator over a finite nonzero b, whose
// quotient is the signed zero a * b.
__device__ __forceinline__ double div_nr(double a, double b) {
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned int eb = (unsigned int)(ub >> 52) & 0x7FFu;
  const unsigned int ea = (unsigned int)(ua >> 52) & 0x7FFu;
  if (eb - 1u >= 2044u || ea - 64u >= 1983u || (int)ea - (int)eb > 1020) {
    if ((ua << 1) == 0 && (ub << 1) != 0 && eb != 0x7FFu) return a * b;
    return a / b;
  }
  // m = b's mantissa in [1, 2) as an FP32 value (leading 24 bits)
  const float mf = __uint_as_float(0x3F800000u | (unsigned int)((ub >> 29) & 0x7FFFFFull));
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(mf));  // ~1/m in (0.5, 1]
  const unsigned int rb = __float_as_uint(r);
  const unsigned long long er = (rb >> 23) & 0xFFu;  // 126 or 127
  // y0 = sign(b) r 2^-(eb - 1023): FP64 exponent field er - 127 + 1023 - (eb - 1023)
  const double y0 = __longlong_as_double((long long)((ub & 0x8000000000000000ull) | ((er + 1919ull - eb) << 52) |
                                                     ((unsigned long long)(rb & 0x7FFFFFu) << 29)));
  const double y1 = fma(y0, fma(-b, y0, 1.0), y0);
  const double q0 = a * y1;
  return fma(y1, fma(-b, q0, a), q0);
}

template <class R>
struct Prec;
template <>
struct Prec<double> {
  static __device__ __forceinline__ double div(double a, double b) { return div_nr(a, b); }
  static __device__ __forceinline__ double clampratio(double r) { return r; }
  static __device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }
};
template <>
struct Prec<float> {
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  // keep tau5/(beta+eps) products finite in FP32
  static __device__ __forceinline__ float clampratio(float r) { return fminf(r, 1e15f); }
  static __device__ __forceinline__ float sqrt_(float a) { return sqrtf(a); }
};

// ---------------------------------------------------------------------------
// Sec. 4.3: incremental-stencil WENO interpolation, left-biased to i+1/2 from
// u_{i-2} .. u_{i+2}.  The right-biased value is the same formula on the
// mirrored stencil.  The weights are computed from the four sub-stencil
// values s0..s3, the smoothness indicators b0, b1, b01, b2, b3 and tau5 by
// wenois_tail; wenois gives them for a general stencil, wenois_c0 /
// wenois_p0 for the two stencils of the deviation form (u_i = 0 in the
// left-biased one, u_{i+1} = 0 in the mirrored one), with the zero terms
// left out.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R wenois_tail(R s0, R s1, R s2, R s3, R b0, R b1, R b01, R b2, R b3, R tau, R eps) {
  const R r01 = Prec<R>::clampratio(Prec<R>::div(tau, b01 + eps));
  const R r0 = Prec<R>::clampratio(Prec<R>::div(tau, b0 + eps));
  const R r1 = Prec<R>::clampratio(Prec<R>::div(tau, b1 + eps));
  const R r2 = Prec<R>::clampratio(Prec<R>::div(tau, b2 + eps));
  const R r3 = Prec<R>::clampratio(Prec<R>::div(tau, b3 + eps));
  const R w0 = R(15.0 / 32.0) * (R(1) + r0 * r01);
  const R w1 = R(5.0 / 32.0) * (R(1) + r1 * r01);
  const R w2 = R(5.0 / 16.0) * (R(1) + r2);
  const R w3 = R(1.0 / 16.0) * (R(1) + r3);
  return Prec<R>::div(w0 * s0 + w1 * s1 + w2 * s2 + w3 * s3, (w0 + w1) + (w2 + w3));
}

// FP64 with one division instead of six: multiplying every eta_k by
// D = b0 b1 b01 b2 b3 (b = beta + eps) leaves the weights
// omega_k = eta_k / sum(eta) unchanged and clears the five ratio divisions:
//   eta0 D = d0 (b0 b01 + tau^2) b1 b2 b3,  eta1 D = d1 (b1 b01 + tau^2) b0 b2 b3,
//   eta2 D = d2 (b2 + tau) b0 b1 b01 b3,    eta3 D = d3 (b3 + tau) b0 b1 b01 b2.
// If the scaled sum leaves the comfortable FP64 range the direct form runs.
template <>
__device__ __forceinline__ double wenois_tail<double>(double s0, double s1, double s2, double s3, double b0,
                                                      double b1, double b01, double b2, double b3, double tau,
                                                      double eps) {
  b0 += eps;
  b1 += eps;
  b01 += eps;
  b2 += eps;
  b3 += eps;
  const double t2 = tau * tau;
  const double p23 = b2 * b3, p01b = (b0 * b1) * b01;
  const double w0 = (15.0 / 32.0) * (b0 * b01 + t2) * (b1 * p23);
  const double w1 = (5.0 / 32.0) * (b1 * b01 + t2) * (b0 * p23);
  const double w2 = (5.0 / 16.0) * (b2 + tau) * (p01b * b3);
  const double w3 = (1.0 / 16.0) * (b3 + tau) * (p01b * b2);
  const double sum = (w0 + w1) + (w2 + w3);
  // 1e-280 < sum < 1e280, as integer compares (sum is a sum of products of non-negative terms)
  const long long sb = __double_as_longlong(sum);
  if (sb > __double_as_longlong(1e-280) && sb < __double_as_longlong(1e280))
    return (w0 * s0 + w1 * s1 + w2 * s2 + w3 * s3) / sum;
  const double r01 = tau / b01;
  const double v0 = (15.0 / 32.0) * (1.0 + (tau / b0) * r01);
  const double v1 = (5.0 / 32.0) * (1.0 + (tau / b1) * r01);
  const double v2 = (5.0 / 16.0) * (1.0 + tau / b2);
  const double v3 = (1.0 / 16.0) * (1.0 + tau / b3);
  return (v0 * s0 + v1 * s1 + v2 * s2 + v3 * s3) / ((v0 + v1) + (v2 + v3));
}

// beta = (13/12) a^2 + (1/4) c^2 for the three-point indicators
template <class R>
__device__ __forceinline__ R beta3(R a, R c) {
  return R(13.0 / 12.0) * a * a + R(0.25) * c * c;
}

template <class R>
__device__ __forceinline__ R wenois(R um2, R um1, R u0, R up1, R up2, R eps) {
  const R s0 = R(0.5) * (u0 + up1);
  const R s1 = R(0.5) * (R(3) * u0 - um1);
  const R s2 = R(0.125) * (R(3) * u0 + R(6) * up1 - up2);
  const R s3 = R(0.125) * (R(3) * um2 - R(10) * um1 + R(15) * u0);
  const R e0 = u0 - up1, e1 = um1 - u0;
  const R b01 = beta3(um1 - R(2) * u0 + up1, um1 - up1);
  const R b2 = beta3(u0 - R(2) * up1 + up2, R(3) * u0 - R(4) * up1 + up2);
  const R b3 = beta3(um2 - R(2) * um1 + u0, um2 - R(4) * um1 + R(3) * u0);
  const R tau = beta3(up2 - R(4) * up1 + R(6) * u0 - R(4) * um1 + um2, up2 - R(2) * up1 + R(2) * um1 - um2);
  return wenois_tail<R>(s0, s1, s2, s3, e0 * e0, e1 * e1, b01, b2, b3, tau, eps);
}

// u0 = 0 (left-biased interpolation of deviations from node i)
template <class R>
__device__ __forceinline__ R wenois_c0(R um2, R um1, R up1, R up2, R eps) {
  const R s0 = R(0.5) * up1;
  const R s1 = R(-0.5) * um1;
  const R s2 = R(0.75) * up1 - R(0.125) * up2;
  const R s3 = R(0.375) * um2 - R(1.25) * um1;
  const R a01 = um1 + up1, c01 = um1 - up1;
  const R b01 = beta3(a01, c01);
  const R b2 = beta3(up2 - R(2) * up1, up2 - R(4) * up1);
  const R b3 = beta3(um2 - R(2) * um1, um2 - R(4) * um1);
  const R tau = beta3((um2 + up2) - R(4) * a01, (up2 - um2) + R(2) * c01);
  return wenois_tail<R>(s0, s1, s2, s3, up1 * up1, um1 * um1, b01, b2, b3, tau, eps);
}

// up1 = 0 (the mirrored, right-biased interpolation of deviations from node i)
template <class R>
__device__ __forceinline__ R wenois_p0(R um2, R um1, R u0, R up2, R eps) {
  const R s0 = R(0.5) * u0;
  const R s1 = R(0.5) * (R(3) * u0 - um1);
  const R s2 = R(0.125) * (R(3) * u0 - up2);
  const R s3 = R(0.125) * (R(3) * um2 - R(10) * um1 + R(15) * u0);
  const R e1 = um1 - u0;
  const R b01 = beta3(um1 - R(2) * u0, um1);
  const R b2 = beta3(u0 + up2, R(3) * u0 + up2);
  const R b3 = beta3(um2 - R(2) * um1 + u0, um2 - R(4) * um1 + R(3) * u0);
  const R tau = beta3((um2 + up2) + R(6) * u0 - R(4) * um1, (up2 - um2) + R(2) * um1);
  return wenois_tail<R>(s0, s1, s2, s3, u0 * u0, e1 * e1, b01, b2, b3, tau, eps);
}

// FP64 forms of the two deviation-form stencils with every smoothness
// indicator, tau5 and eps scaled by 4: the weights depend only on ratios
// of these quantities and on products with equal numbers of them, so they
// are unchanged in exact arithmetic, and 4 beta = (13/3) a^2 + c^2 takes
// the eps addition into an FMA.  e4 = 4 eps.
__device__ __forceinline__ double beta3x4(double a, double c, double e4) {
  return fma((13.0 / 3.0) * a, a, fma(c, c, e4));
}

// IS weights and interpolated value from the scaled indicators (eps
// already included), one division.  With the linear weights
// d = (15, 5, 10, 2)/32 and D = b0 b1 b01 b2 b3, the scaled weights
// eta_k D / (5/32) factor as
//   (b2 b3) [3 (b0 b01 + tau^2) b1 | (b1 b01 + tau^2) b0]   for k = 0, 1,
//   (b0 b1 b01) [2 (b2 + tau) b3 | 0.4 (b3 + tau) b2]       for k = 2, 3;
// the factors 3 and 2 are carried by the sub-stencil values: s0x3 = 3 s0,
// s2x2 = 2 s2 (the callers form them at no extra cost).
__device__ __forceinline__ double wenois_tail_x4(double s0x3, double s1, double s2x2, double s3, double b0,
                                                 double b1, double b01, double b2, double b3, double tau) {
  const double t2 = tau * tau;
  const double Q = b2 * b3, Pb = (b0 * b1) * b01;
  const double A0 = fma(b0, b01, t2) * b1;  // weight 0 / 3
  const double A1 = fma(b1, b01, t2) * b0;  // weight 1
  const double B2 = (b2 + tau) * b3;        // weight 2 / 2
  const double B3 = 0.4 * (b3 + tau) * b2;  // weight 3
  const double num = fma(Q, fma(A0, s0x3, A1 * s1), Pb * fma(B2, s2x2, B3 * s3));
  const double den = fma(Q, fma(3.0, A0, A1), Pb * fma(2.0, B2, B3));
  // 1e-280 < den < 1e280, as integer compares (den is a sum of products of non-negative terms)
  const long long db = __double_as_longlong(den);
  if (db > __double_as_longlong(1e-280) && db < __double_as_longlong(1e280)) return div_nr(num, den);
  // outside that range: the weights from the ratios tau / b, as printed
  const double r01 = tau / b01;
  const double v0 = 1.0 + (tau / b0) * r01, v1 = 1.0 + (tau / b1) * r01;
  const double v2 = 1.0 + tau / b2, v3 = 1.0 + tau / b3;
  return ((5.0 / 32.0) * (v0 * s0x3 + v1 * s1 + v2 * s2x2) + (1.0 / 16.0) * v3 * s3) /
         ((15.0 / 32.0) * v0 + (5.0 / 32.0) * v1 + (5.0 / 16.0) * v2 + (1.0 / 16.0) * v3);
}

// u0 = 0: as wenois_c0, indicators scaled by 4
__device__ __forceinline__ double wenois_c0_x4(double um2, double um1, double up1, double up2, double e4) {
  const double s0x3 = 1.5 * up1;                  // 3 s0
  const double s1 = -0.5 * um1;
  const double s2x2 = 1.5 * up1 - 0.25 * up2;     // 2 s2
  const double s3 = 0.375 * um2 - 1.25 * um1;
  const double a01 = um1 + up1, c01 = um1 - up1;
  const double b01 = beta3x4(a01, c01, e4);
  const double b2 = beta3x4(up2 - 2.0 * up1, up2 - 4.0 * up1, e4);
  const double b3 = beta3x4(um2 - 2.0 * um1, um2 - 4.0 * um1, e4);
  const double ta = (um2 + up2) - 4.0 * a01, tc = (up2 - um2) + 2.0 * c01;
  const double tau = fma((13.0 / 3.0) * ta, ta, tc * tc);
  return wenois_tail_x4(s0x3, s1, s2x2, s3, fma(4.0 * up1, up1, e4), fma(4.0 * um1, um1, e4), b01, b2, b3, tau);
}

// up1 = 0: as wenois_p0, indicators scaled by 4
__device__ __forceinline__ double wenois_p0_x4(double um2, double um1, double u0, double up2, double e4) {
  const double s0x3 = 1.5 * u0;                   // 3 s0
  const double s1 = 0.5 * (3.0 * u0 - um1);
  const double s2x2 = 0.25 * (3.0 * u0 - up2);    // 2 s2
  const double s3 = 0.125 * (3.0 * um2 - 10.0 * um1 + 15.0 * u0);
  const double e1 = um1 - u0;
  const double b01 = beta3x4(um1 - 2.0 * u0, um1, e4);
  const double b2 = beta3x4(u0 + up2, 3.0 * u0 + up2, e4);
  const double b3 = beta3x4(um2 - 2.0 * um1 + u0, um2 - 4.0 * um1 + 3.0 * u0, e4);
  const double ta = (um2 + up2) + 6.0 * u0 - 4.0 * um1, tc = (up2 - um2) + 2.0 * um1;
  const double tau = fma((13.0 / 3.0) * ta, ta, tc * tc);
  return wenois_tail_x4(s0x3, s1, s2x2, s3, fma(4.0 * u0, u0, e4), fma(4.0 * e1, e1, e4), b01, b2, b3, tau);
}

// ---------------------------------------------------------------------------
// Sec. 3.1-3.2: HLLC flux in direction DIR from two states given by their
// conservative vector, velocity, pressure, density and sound speed.
// Returns G (nf components, alpha flux last) and s* (= u-hat).
// The star-state jumps W*_K - W_K are evaluated in a cancellation-free form
// (algebraically identical to the paper's W*_K minus W_K), with
// chi - 1 = (s* - u_K)/(s_K - s*):
//   d(a_k rho_k) = (chi-1) a_k rho_k,   d(rho u_n) = rho s_K (chi-1),
//   d(rho u_t)   = (chi-1) rho u_t,
//   dE = (chi-1)(E + p) + chi rho s* (s* - u_K).
// ---------------------------------------------------------------------------
template <int NDIM, int DIR, class R>
__device__ __forceinline__ void hllc(const R *WL, const R *vL, R pL, R rL, R cL, const R *WR,
                                     const R *vR, R pR, R rR, R cR, R *G, R &sstar) {
  constexpr int NF = NDIM + 4, E = 2 + NDIM, A = 3 + NDIM;
  const R uL = vL[DIR], uR = vR[DIR];
  const R ubar = R(0.5) * (uL + uR), cbar = R(0.5) * (cL + cR);
  const R sL = fmin(ubar - cbar, uL - cL);
  const R sR = fmax(ubar + cbar, uR + cR);
  const R mL = rL * (sL - uL), mR = rR * (sR - uR);
  const R ss = Prec<R>::div(pR - pL + mL * uL - mR * uR, mL - mR);
  sstar = ss;
  // One side's flux F_K + s_(-/+) (W*_K - W_K); at s* = 0 the mean of both.
  R GL[NF], GR[NF];
  bool needL, needR;
  if constexpr (sizeof(R) == 8) {
    needL = !negative64(ss);
    needR = !positive64(ss);
  } else {
    needL = !(ss < R(0));
    needR = !(ss > R(0));
  }
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    if ((side == 0 && !needL) || (side == 1 && !needR)) continue;
    const R *W = side ? WR : WL;
    const R *v = side ? vR : vL;
    const R p = side ? pR : pL;
    const R rho = side ? rR : rL;
    const R u = side ? uR : uL;
    const R sK = side ? sR : sL;
    const R sw = side ? fmax(R(0), sR) : fmin(R(0), sL);
    R *Gs = side ? GR : GL;
    const R chim1 = Prec<R>::div(ss - u, sK - ss);
    Gs[0] = W[0] * u + sw * (chim1 * W[0]);
    Gs[1] = W[1] * u + sw * (chim1 * W[1]);
#pragma unroll
    for (int j = 0; j < NDIM; ++j) {
      const R m = W[2 + j];
      const R dm = (j == DIR) ? rho * sK * chim1 : chim1 * (rho * v[j]);
      Gs[2 + j] = m * u + ((j == DIR) ? p : R(0)) + sw * dm;
    }
    const R dE = chim1 * (W[E] + p) + (R(1) + chim1) * rho * ss * (ss - u);
    Gs[E] = (W[E] + p) * u + sw * dE;
    Gs[A] = W[A] * ss;
  }
  if (needL && needR) {
#pragma unroll
    for (int q = 0; q < NF; ++q) G[q] = R(0.5) * (GL[q] + GR[q]);
  } else if (needL) {
#pragma unroll
    for (int q = 0; q < NF; ++q) G[q] = GL[q];
  } else {
#pragma unroll
    for (int q = 0; q < NF; ++q) G[q] = GR[q];
  }
}

// Reference node state for the deviation form (mixed path): the large
// quantities of node i, rounded to R; they only ever multiply deviations or
// enter quantities needed to relative precision (wave speeds, star jumps).
template <int NDIM, class R>
struct RefNode {
  R r1, r2, rho, u[NDIM], p, Ep, a1;  // a1r1, a2r2, rho, velocity, p, E + p, alpha1
};

// One state K described by its deviation from the reference node:
// (d a1r1, d a2r2, d u_1..d u_ndim, d p, d alpha1) and its sound speed.
// HLLC flux deviation dG = G^HLLC(L, R) - G(ref) (Sec. 3.2) and s*.  The
// physical-flux deviations F(ref + d) - F(ref) are expanded exactly, e.g.
//   d(rho u_n^2 + p) = d rho u_n,K^2 + rho_ref d u_n (2 u_n,ref + d u_n) + d p,
//   d((E + p) u_n)   = (dE + dp) u_n,K + (E + p)_ref d u_n,
//   dE = dp Gamma_K + (p_ref (r1 - r2) + q1) d alpha1
//        + (d rho |u_K|^2 + rho_ref sum_j d u_j (2 u_j,ref + d u_j)) / 2,
// so that FP32 rounding scales with the deviations, not with |G|.
template <int NDIM, int DIR, class R>
__device__ __forceinline__ void hllc_dev(const RefNode<NDIM, R> &ref, const EosConst &eos, const R *dL, R cL,
                                         const R *dR, R cR, R *dG, R &sstar) {
  constexpr int NF = NDIM + 4, E = 2 + NDIM, A = 3 + NDIM;
  const R *dv[2] = {dL, dR};
  R rho[2], un[2], a1r1[2], a2r2[2], al[2], pdev[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    a1r1[k] = ref.r1 + dv[k][0];
    a2r2[k] = ref.r2 + dv[k][1];
    rho[k] = a1r1[k] + a2r2[k];
    un[k] = ref.u[DIR] + dv[k][2 + DIR];
    pdev[k] = dv[k][E];
    al[k] = ref.a1 + dv[k][A];
  }
  const R cK[2] = {cL, cR};
  const R ubar = R(0.5) * (un[0] + un[1]), cbar = R(0.5) * (cL + cR);
  const R sL = fmin(ubar - cbar, un[0] - cL);
  const R sR = fmax(ubar + cbar, un[1] + cR);
  const R mL = rho[0] * (sL - un[0]), mR = rho[1] * (sR - un[1]);
  const R ss = Prec<R>::div(pdev[1] - pdev[0] + mL * un[0] - mR * un[1], mL - mR);
  sstar = ss;
  const R rdiff = (R)eos.drf, q1 = (R)eos.q1f;
  // One side's flux deviation F_K - G(ref) + s_(-/+) (W*_K - W_K) into Gk;
  // the side is a compile-time constant, so no array is indexed at run time.
  auto side_flux = [&](auto kc, R *Gk) {
    constexpr int k = decltype(kc)::value;
    const R *d = k ? dR : dL;
    const R u = un[k];
    const R sK = k ? sR : sL;
    const R sw = k ? fmax(R(0), sR) : fmin(R(0), sL);
    const R chim1 = Prec<R>::div(ss - u, sK - ss);
    const R drho = d[0] + d[1];
    // velocity of K and |u_K|^2 deviation
    R uK[NDIM], du2 = R(0), uk2 = R(0);
#pragma unroll
    for (int j = 0; j < NDIM; ++j) {
      uK[j] = ref.u[j] + d[2 + j];
      du2 += d[2 + j] * (R(2) * ref.u[j] + d[2 + j]);
      uk2 += uK[j] * uK[j];
    }
    const R GammaK = (R)eos.r2f + rdiff * al[k];
    const R dE = d[E] * GammaK + (ref.p * rdiff + q1) * d[A] + R(0.5) * (drho * uk2 + ref.rho * du2);
    const R EpK = ref.Ep + dE + d[E];  // (E + p)_K
    // physical-flux deviations
    Gk[0] = d[0] * u + ref.r1 * d[2 + DIR] + sw * (chim1 * a1r1[k]);
    Gk[1] = d[1] * u + ref.r2 * d[2 + DIR] + sw * (chim1 * a2r2[k]);
#pragma unroll
    for (int j = 0; j < NDIM; ++j) {
      R dF;
      if (j == DIR)
        dF = drho * u * u + ref.rho * d[2 + DIR] * (R(2) * ref.u[DIR] + d[2 + DIR]) + d[E];
      else
        dF = drho * uK[j] * u + ref.rho * (d[2 + j] * u + ref.u[j] * d[2 + DIR]);
      const R dm = (j == DIR) ? rho[k] * sK * chim1 : chim1 * (rho[k] * uK[j]);
      Gk[2 + j] = dF + sw * dm;
    }
    const R dEstar = chim1 * EpK + (R(1) + chim1) * rho[k] * ss * (ss - u);
    Gk[E] = (dE + d[E]) * u + ref.Ep * d[2 + DIR] + sw * dEstar;
    Gk[A] = al[k] * ss - ref.a1 * ref.u[DIR];
  };
  const bool needL = !(ss < R(0)), needR = !(ss > R(0));
  if (needL && needR) {  // s* = 0: the mean of both sides
    R GL[NF], GR[NF];
    side_flux(std::integral_constant<int, 0>{}, GL);
    side_flux(std::integral_constant<int, 1>{}, GR);
#pragma unroll
    for (int q = 0; q < NF; ++q) dG[q] = R(0.5) * (GL[q] + GR[q]);
  } else if (needL) {
    side_flux(std::integral_constant<int, 0>{}, dG);
  } else {
    side_flux(std::integral_constant<int, 1>{}, dG);
  }
}

// ---------------------------------------------------------------------------
// Sec. 2: mixture EOS helpers (FP64).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double mixGamma(const EosConst &e, double a1) { return fma(a1, e.dr, e.r2); }
__device__ __forceinline__ double mixPi(const EosConst &e, double a1) { return a1 * e.q1; }
// pbar = Pi (gbar - 1)/gbar = Pi / (Gamma + 1)
__device__ __forceinline__ double mixPinf(const EosConst &e, double a1) {
  return mixPi(e, a1) / (mixGamma(e, a1) + 1.0);
}

// rho*ctilde^2 = rho e - pbar (Sec. 5.1 helper) of a conservative state.
template <int NDIM>
__device__ __forceinline__ double rho_ct2(const EosConst &e, const double *W) {
  constexpr int E = 2 + NDIM, A = 3 + NDIM;
  const double rho = W[0] + W[1];
  double m2 = 0.0;
#pragma unroll
  for (int j = 0; j < NDIM; ++j) m2 = fma(W[2 + j], W[2 + j], m2);
  return W[E] - 0.5 * m2 / rho - mixPinf(e, W[A]);
}

// "rho ctilde^2 < eps" decided without divisions: for rho > 0 and
// Gamma + 1 > 0, multiply E - m^2/(2 rho) - Pi/(Gamma+1) < eps through by
// rho (Gamma + 1).  Any other state uses the quotient form.  Every operation
// is explicitly rounded (no contraction left to the compiler), so all call
// sites take the same decision for the same state, also where rounding
// decides it.
template <int NDIM>
__device__ __forceinline__ bool rct2_below(const EosConst &e, const double *W, double eps) {
  constexpr int E = 2 + NDIM, A = 3 + NDIM;
  const double rho = W[0] + W[1];
  const double G1 = mixGamma(e, W[A]) + 1.0;
  if (!positive64(rho) || !positive64(G1)) return rho_ct2<NDIM>(e, W) < eps;
  double m2 = 0.0;
#pragma unroll
  for (int j = 0; j < NDIM; ++j) m2 = fma(W[2 + j], W[2 + j], m2);
  const double s = __fma_rn(__dsub_rn(W[E], eps), rho, __dmul_rn(-0.5, m2));
  return negative64(__fma_rn(s, G1, -__dmul_rn(mixPi(e, W[A]), rho)));
}

// theta solving (1-theta) fA + theta fB = eps with the paper's three cases:
// false for theta = 1 (nothing to blend), else true with th set.  The
// threshold tests are integer compares (eps >= 0).
__device__ __forceinline__ bool lim_theta(double fA, double fB, double eps, double &th) {
  if (below64(fA, eps)) {
    th = 0.0;
    return true;
  }
  if (below64(fB, eps)) {
    th = (fA - eps) / (fA - fB);
    return true;
  }
  return false;
}

// The same three cases for rho ctilde^2, with the quotient evaluated only
// when a blend is needed.
template <int NDIM>
__device__ __forceinline__ bool lim_theta_rct(const EosConst &e, const double *A, const double *B, double eps,
                                              double &th) {
  if (rct2_below<NDIM>(e, A, eps)) {
    th = 0.0;
    return true;
  }
  if (!rct2_below<NDIM>(e, B, eps)) return false;
  const double fA = rho_ct2<NDIM>(e, A);
  th = (fA - eps) / (fA - rho_ct2<NDIM>(e, B));
  return true;
}

template <int NDIM>
__device__ __forceinline__ double lim_quantity(const double *W, int which) {
  constexpr int A = 3 + NDIM;
  switch (which) {
    case 0: return W[0];
    case 1: return W[1];
    case 2: return W[A];
    default: return 1.0 - W[A];
  }
}

// Hard-switch test of Secs. 5.1-5.2: a tested quantity below its
// hard-switch tolerance.
template <int NDIM>
__device__ __forceinline__ bool hard_fail(const EosConst &e, const LimTol &t, const double *X) {
  constexpr int A = 3 + NDIM;
  return below64(X[0], t.hs_ar) || below64(X[1], t.hs_ar) || below64(X[A], t.hs_a) ||
         below64(1.0 - X[A], t.hs_a) || rct2_below<NDIM>(e, X, t.hs_rc);
}

// Sec. 5.1, Algorithms 1-3 + hard switch: limit Wt toward the node state Wn.
// Returns bit 0 = some theta < 1, bit 1 = hard switch.
template <int NDIM>
__device__ int interp_limit(const EosConst &e, const LimTol &t, const double *Wn, double *Wt) {
  constexpr int NF = NDIM + 4;
  int flags = 0;
  bool any = false;  // some threshold test fired
#pragma unroll 1
  for (int which = 0; which < 5; ++which) {
    double th = 1.0;
    bool lim;
    if (which < 4) {
      const double eps = which < 2 ? t.eps_ar : t.eps_a;
      lim = lim_theta(lim_quantity<NDIM>(Wn, which), lim_quantity<NDIM>(Wt, which), eps, th);
    } else {
      lim = lim_theta_rct<NDIM>(e, Wn, Wt, t.eps_rc, th);
    }
    any = any || lim;
    if (lim && th < 1.0) {
      flags |= 1;
#pragma unroll
      for (int q = 0; q < NF; ++q) Wt[q] = (1.0 - th) * Wn[q] + th * Wt[q];
    }
  }
  // Wt passed every threshold test unblended: each quantity is >= its eps
  // (rounding is monotone), hence >= its hard-switch tolerance
  if ((any || !t.hs_implied) && hard_fail<NDIM>(e, t, Wt)) {
    flags |= 2;
#pragma unroll
    for (int q = 0; q < NF; ++q) Wt[q] = Wn[q];
  }
  return flags;
}

// Sec. 5.2, Algorithms 4-6 + hard switch at one midpoint.  Gm/Gp: high-order
// split fluxes in, limited fluxes out.  Returns bit 0 = some theta < 1,
// bit 1 = hard switch.
template <int NDIM>
__device__ int flux_limit(const EosConst &e, const LimTol &t, const double *Wi, const double *Wi1,
                          const double *Fi, const double *Fi1, const double *GHm, const double *GHp,
                          double lam, double *Gm, double *Gp) {
  constexpr int NF = NDIM + 4;
  const double l2 = 2.0 * lam;
  double Ap[NF], Am[NF], Bp[NF], Bm[NF];
#pragma unroll
  for (int q = 0; q < NF; ++q) {
    Ap[q] = Wi[q] - l2 * (GHm[q] - Fi[q]);
    Am[q] = Wi1[q] + l2 * (GHp[q] - Fi1[q]);
    Bp[q] = Wi[q] - l2 * (Gm[q] - Fi[q]);
    Bm[q] = Wi1[q] + l2 * (Gp[q] - Fi1[q]);
  }
  int flags = 0;
  bool any = false;  // some threshold test fired
#pragma unroll 1
  for (int which = 0; which < 5; ++which) {
    double thp = 1.0, thm = 1.0;
    bool lp, lm;
    if (which < 4) {
      const double eps = which < 2 ? t.eps_ar : t.eps_a;
      lp = lim_theta(lim_quantity<NDIM>(Ap, which), lim_quantity<NDIM>(Bp, which), eps, thp);
      lm = lim_theta(lim_quantity<NDIM>(Am, which), lim_quantity<NDIM>(Bm, which), eps, thm);
    } else {
      lp = lim_theta_rct<NDIM>(e, Ap, Bp, t.eps_rc, thp);
      lm = lim_theta_rct<NDIM>(e, Am, Bm, t.eps_rc, thm);
    }
    any = any || lp || lm;
    const double th = (lp || lm) ? fmin(thp, thm) : 1.0;
    if ((lp || lm) && th < 1.0) {
      flags |= 1;
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        Gp[q] = (1.0 - th) * GHp[q] + th * Gp[q];
        Gm[q] = (1.0 - th) * GHm[q] + th * Gm[q];
        Bp[q] = Wi[q] - l2 * (Gm[q] - Fi[q]);
        Bm[q] = Wi1[q] + l2 * (Gp[q] - Fi1[q]);
      }
    }
  }
  // as in interp_limit: unblended half states that passed every test
  if ((any || !t.hs_implied) && (hard_fail<NDIM>(e, t, Bp) || hard_fail<NDIM>(e, t, Bm))) {
    flags |= 2;
#pragma unroll
    for (int q = 0; q < NF; ++q) {
      Gp[q] = GHp[q];
      Gm[q] = GHm[q];
    }
  }
  return flags;
}

// ---------------------------------------------------------------------------
// FP32 certification of the limiter tests of the FP64 sweeps.  Where every
// threshold test of Algorithms 1-6 passes, the limiters leave states and
// fluxes as they are (theta = 1).  The functions below decide that in FP32
// from truncated images of the FP64 operands, with an error bound that
// covers the truncation, the FP32 evaluation and the FP64 evaluation of the
// exact test: a test certified here passes in FP64 as well, so a certified
// midpoint gets exactly the FP64 limiters' result.  Whatever is not
// certified goes through interp_limit / flux_limit.
// ---------------------------------------------------------------------------

// FP32 image of an FP64 value from its high word alone (integer operations
// only): sign, exponent and the leading 20 mantissa bits, truncated toward
// zero, so |x - t(x)| < 2^-20 |x| and |t(x)| <= |x|.  A value below the
// FP32 normal range maps to 0 (absolute error below 2^-126: the bounds below
// add CTINY for it); a value at or above 2^128 or not finite maps to a NaN,
// which fails every certification test.
__device__ __forceinline__ float trunc32(double x) {
  const unsigned int hi = (unsigned int)__double2hiint(x);
  const unsigned int mag = hi & 0x7FFFFFFFu;
  // FP64 exponent field in [897, 1150] <=> FP32 exponent field in [1, 254]
  if (mag - 0x38100000u < 0x0FE00000u) return __uint_as_float((hi & 0x80000000u) | ((mag - 0x38000000u) << 3));
  return mag < 0x38100000u ? 0.0f : __uint_as_float(0x7FC00000u);
}
constexpr float CTINY = 2.350988701644575e-38f;  // 2^-125: twice trunc32's absolute error on tiny values

// Error allowance 2^-18 m for a quantity of operand magnitude m: at least
// three times the truncation error (2^-20), the FP32 roundings of the short
// expressions below and the FP64 roundings of the exact tests together.
__device__ __forceinline__ float cmargin(float m) { return 3.814697265625e-06f * m; }

// Certify rho ctilde^2 = E - |m|^2 / (2 rho) - Pi / (Gamma + 1) >= eps (Sec.
// 2) for a conservative state whose every component X_f lies within d[f] of
// the FP32 value x[f], alpha certified inside [0, 1].  Errors propagated:
// rho, the kinetic energy (through m and rho), pbar (through alpha, with
// |d pbar / d alpha| = q1 (r2 + 1) / (Gamma + 1)^2 <= |q1| (|r2| + 1) on
// [0, 1]; through the FP32 constants and Gamma + 1, whose rounding is
// bounded by the magnitudes of its two terms) and the FP32 evaluation.
template <int NDIM>
__device__ __forceinline__ bool rct2_cert(const EosConst &e, const float *x, const float *d, float eps) {
  constexpr int E = 2 + NDIM, A = 3 + NDIM;
  const float rho = x[0] + x[1];
  const float drho = d[0] + d[1] + cmargin(fabsf(rho));
  const float rlo = rho - drho;
  if (!(rlo > 0.0f) || !(rho < 1e30f)) return false;
  float m2 = 0.0f, dm2 = 0.0f;
#pragma unroll
  for (int j = 0; j < NDIM; ++j) {
    m2 = fmaf(x[2 + j], x[2 + j], m2);
    dm2 = fmaf(2.0f * fabsf(x[2 + j]) + d[2 + j], d[2 + j], dm2);
  }
  const float ke = 0.5f * __fdividef(m2, rho);
  const float dke = 0.5f * __fdividef(dm2, rlo) + __fdividef(ke * drho, rlo) + cmargin(ke);
  const float al = x[A];
  const float g0 = e.r2f + 1.0f, gd = e.drf * al;
  const float G1 = g0 + gd;  // Gamma + 1 >= 1 for alpha in [0, 1]
  if (!(G1 > 0.5f) || !(G1 < 1e30f)) return false;
  const float pb = __fdividef(e.q1f * al, G1);
  const float dpb = fabsf(e.q1f) * (fabsf(e.r2f) + 1.0f) * d[A] +
                    cmargin(pb * (1.0f + __fdividef(g0 + fabsf(gd), G1)));
  const float v = x[E] - ke - pb;
  return v - (d[E] + dke + dpb + cmargin(fabsf(x[E]) + ke + pb)) >= eps;
}

// The five threshold tests of a conservative FP64 state W at their
// tolerances (Algorithms 1-3, the quantities of node or interpolated state),
// exactly as interp_limit decides them, with rho ctilde^2 certified in FP32
// first and tested in FP64 only where that fails.
template <int NDIM>
__device__ __forceinline__ bool state_passes(const EosConst &e, const LimTol &t, const double *W) {
  constexpr int NF = NDIM + 4, A = 3 + NDIM;
  if (below64(W[0], t.eps_ar) || below64(W[1], t.eps_ar) || below64(W[A], t.eps_a) ||
      below64(1.0 - W[A], t.eps_a))
    return false;
  float x[NF], d[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    x[f] = trunc32(W[f]);
    d[f] = cmargin(fabsf(x[f])) + CTINY;
  }
  return rct2_cert<NDIM>(e, x, d, t.cert_rc) || !rct2_below<NDIM>(e, W, t.eps_rc);
}

// An FP32 value with a bound on its distance to the exact value it stands
// for (running error analysis).  An operation's bound is the propagated
// bounds of its operands plus 2^-22 of the result for its own rounding (at
// least twice an FP32 rounding); a division needs its denominator bounded
// away from zero.  The bounds are computed in FP32 themselves; the slack
// of every term (2x or more) covers their own rounding.
struct EF {
  float v, e;
};
constexpr float EF_U = 2.384185791015625e-07f;  // 2^-22
// from an FP64 value: the truncated image, within 2^-20 |x| <= 2^-19 |v|
// (within 2^-126 for a value below the FP32 normal range)
__device__ __forceinline__ EF ef(double x) {
  const float v = trunc32(x);
  return {v, 1.9073486328125e-06f * fabsf(v) + CTINY};
}
__device__ __forceinline__ EF operator+(EF a, EF b) {
  const float v = a.v + b.v;
  return {v, a.e + b.e + EF_U * fabsf(v)};
}
__device__ __forceinline__ EF operator-(EF a, EF b) {
  const float v = a.v - b.v;
  return {v, a.e + b.e + EF_U * fabsf(v)};
}
__device__ __forceinline__ EF operator*(EF a, EF b) {
  const float v = a.v * b.v;
  return {v, fabsf(a.v) * b.e + fabsf(b.v) * a.e + a.e * b.e + EF_U * fabsf(v)};
}
// exact constants: 0.5 and 1 times a value
__device__ __forceinline__ EF half(EF a) { return {0.5f * a.v, 0.5f * a.e}; }
__device__ __forceinline__ EF efmin(EF a, EF b) { return {fminf(a.v, b.v), fmaxf(a.e, b.e)}; }
__device__ __forceinline__ EF efmax(EF a, EF b) { return {fmaxf(a.v, b.v), fmaxf(a.e, b.e)}; }
// a / b = q: |A/B - q| <= (ea + |q| eb) / (|b| - eb) plus the rounding of
// the approximate division (2 ulp); ok cleared unless |b| - eb > 0 and b is
// inside the approximate division's range
__device__ __forceinline__ EF operator/(EF a, EF b) {
  const float den = fabsf(b.v) - b.e;
  const bool good = den > 0.0f && fabsf(b.v) < 1e30f;
  const float q = __fdividef(a.v, b.v);
  return {q, good ? __fdividef(a.e + fabsf(q) * b.e, den) + 2.0f * EF_U * fabsf(q) : __int_as_float(0x7FC00000)};
}

// First-order HLLC flux G^HLLC(W_i, W_{i+1}) (Sec. 3.2, the formulas of
// hllc above) in FP32 with error bounds, from the FP64 node states W, their
// velocities, pressures and sound speeds.  gH / eH: the shared components
// (f < A), then the alpha components of G^{HLLC,-} and G^{HLLC,+} at A and
// A + 1.  The bounds cover whatever the FP64 flux computes:
// - where |s*| exceeds its bound, the FP64 flux takes the same star state;
// - otherwise it takes either star state or their mean (at s* = 0), and
//   the mean of both FP32 side fluxes with half their difference added to
//   the bound covers all three;
// - the alpha components (alpha_K - alpha_i) s*, (alpha_K - alpha_{i+1}) s*
//   take the alpha differences from FP64, so that their bounds scale with
//   the jump in alpha, plus an allowance for the FP64 path's own rounding
//   of alpha_K s* - alpha_i s*.
// Returns false where a denominator is not bounded away from zero or a
// bound is not finite.
template <int NDIM, int DIR>
__device__ __forceinline__ bool hllc1_bound32(const double *WL, const double *vL, double pL, double cL,
                                              const double *WR, const double *vR, double pR, double cR, float *gH,
                                              float *eH) {
  constexpr int NF = NDIM + 4, E = 2 + NDIM, A = 3 + NDIM;
  const EF uL = ef(vL[DIR]), uR = ef(vR[DIR]), cl = ef(cL), cr = ef(cR);
  const EF rL = ef(WL[0]) + ef(WL[1]), rR = ef(WR[0]) + ef(WR[1]);
  const EF pl = ef(pL), pr = ef(pR);
  const EF ubar = half(uL + uR), cbar = half(cl + cr);
  const EF sL = efmin(ubar - cbar, uL - cl);
  const EF sR = efmax(ubar + cbar, uR + cr);
  const EF mL = rL * (sL - uL), mR = rR * (sR - uR);
  const EF ss = (pr - pl + mL * uL - mR * uR) / (mL - mR);
  if (!(ss.e < 1e30f)) return false;  // also a NaN
  // one side's flux F_K + s_(-/+) (W*_K - W_K), shared components
  auto side_flux = [&](bool right, EF *G) {
    const double *W = right ? WR : WL;
    const double *v = right ? vR : vL;
    const EF u = right ? uR : uL, sK = right ? sR : sL, p = right ? pr : pl, rho = right ? rR : rL;
    const EF sw = right ? EF{fmaxf(0.0f, sR.v), sR.e} : EF{fminf(0.0f, sL.v), sL.e};
    const EF chim1 = (ss - u) / (sK - ss);
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const EF w = ef(W[f]);
      G[f] = w * u + sw * (chim1 * w);
    }
#pragma unroll
    for (int j = 0; j < NDIM; ++j) {
      const EF m = ef(W[2 + j]);
      const EF dm = (j == DIR) ? (rho * sK) * chim1 : chim1 * (rho * ef(v[j]));
      G[2 + j] = (j == DIR) ? m * u + p + sw * dm : m * u + sw * dm;
    }
    const EF Ep = ef(W[E]) + p;
    const EF dE = chim1 * Ep + ((EF{1.0f, 0.0f} + chim1) * rho) * (ss * (ss - u));
    G[E] = Ep * u + sw * dE;
  };
  // alpha jump between the nodes, from FP64; the FP64 path rounds
  // alpha_K s* and alpha_K s* - alpha_i s*: 2^-51 (|alpha_K| + |alpha_i|) |s*|
  const EF da = ef(WR[A] - WL[A]);
  const float aflux = 4.440892098500626e-16f * (fabsf(trunc32(WL[A])) + fabsf(trunc32(WR[A])) + 1.0f) *
                      (fabsf(ss.v) + ss.e);
  EF G[NF - 1];
  EF Gm, Gp;  // (alpha_K - alpha_i) s*, (alpha_K - alpha_{i+1}) s*
  if (fabsf(ss.v) > ss.e) {
    const bool right = ss.v < 0.0f;
    side_flux(right, G);
    Gm = right ? da * ss : EF{0.0f, 0.0f};
    Gp = right ? EF{0.0f, 0.0f} : EF{0.0f, 0.0f} - da * ss;
  } else {
    EF GL[NF - 1], GR[NF - 1];
    side_flux(false, GL);
    side_flux(true, GR);
#pragma unroll
    for (int f = 0; f < NF - 1; ++f) {
      const float v = 0.5f * (GL[f].v + GR[f].v);
      G[f] = {v, 0.5f * fabsf(GL[f].v - GR[f].v) + GL[f].e + GR[f].e + EF_U * fabsf(v)};
    }
    const EF t = da * ss;  // Gm is 0 or t or t/2, Gp is -t or 0 or -t/2
    Gm = {0.5f * t.v, 0.5f * fabsf(t.v) + t.e};
    Gp = {-0.5f * t.v, 0.5f * fabsf(t.v) + t.e};
  }
  bool ok = true;
#pragma unroll
  for (int f = 0; f < A; ++f) {
    gH[f] = G[f].v;
    eH[f] = G[f].e;
    ok = ok && eH[f] < 1e30f;  // false for a NaN bound too
  }
  gH[A] = Gm.v;
  eH[A] = Gm.e + aflux;
  gH[A + 1] = Gp.v;
  eH[A + 1] = Gp.e + aflux;
  return ok && eH[A] < 1e30f && eH[A + 1] < 1e30f;
}

// Certify that flux_limit leaves G^-, G^+ unchanged at a midpoint: the four
// half states W_i - 2 lam (G^{HLLC,-} - F_i), W_{i+1} + 2 lam (G^{HLLC,+} -
// F_{i+1}), W_i - 2 lam (G^- - F_i), W_{i+1} + 2 lam (G^+ - F_{i+1}) (Sec.
// 5.2; F^alpha = 0) pass all five threshold tests.  gH / eH: the first-order
// flux in FP32 with error bounds, laid out as hllc1_bound32 gives it; Gh:
// the FP64 high-order flux (shared components, f < A), GmA / GpA the alpha
// components of G^- and G^+.  l2f: 2 lam in FP32.
template <int NDIM>
__device__ __forceinline__ bool flux_certified(const EosConst &e, const LimTol &t, float l2f, const double *Wi,
                                               const double *Wi1, const double *Fi, const double *Fi1,
                                               const float *gH, const float *eH, const double *Gh, double GmA,
                                               double GpA) {
  constexpr int NF = NDIM + 4, A = 3 + NDIM;
  const float tiny = CTINY * (1.0f + 2.0f * l2f);  // operands truncated to 0
#pragma unroll
  for (int st = 0; st < 4; ++st) {
    const bool right = st & 1;  // W_{i+1} + 2 lam (.) else W_i - 2 lam (.)
    const bool first = st < 2;
    const double *W = right ? Wi1 : Wi;
    const double *F = right ? Fi1 : Fi;
    const float sl = right ? l2f : -l2f;
    float x[NF], d[NF];
#pragma unroll
    for (int f = 0; f < A; ++f) {
      const float w = trunc32(W[f]), fl = trunc32(F[f]);
      const float g = first ? gH[f] : trunc32(Gh[f]);
      x[f] = fmaf(sl, g - fl, w);
      d[f] = cmargin(fabsf(w) + l2f * (fabsf(g) + fabsf(fl))) + (first ? 1.001f * l2f * eH[f] : 0.0f) + tiny;
    }
    const float wa = trunc32(W[A]);
    const float ga = first ? gH[A + (right ? 1 : 0)] : trunc32(right ? GpA : GmA);
    const float eg = (first ? 1.001f * l2f * eH[A + (right ? 1 : 0)] : 0.0f) + tiny;
    x[A] = fmaf(sl, ga, wa);
    d[A] = cmargin(fabsf(wa) + l2f * fabsf(ga)) + eg;
    // 1 - alpha from 1 - W_alpha formed in FP64 (exact for W_alpha >= 1/2),
    // so that its bound scales with 1 - alpha, not with 1
    const float om_w = trunc32(1.0 - W[A]);
    const float om = fmaf(-sl, ga, om_w);
    if (!(x[0] - d[0] >= t.cert_ar && x[1] - d[1] >= t.cert_ar && x[A] - d[A] >= t.cert_a &&
          om - (cmargin(fabsf(om_w) + l2f * fabsf(ga)) + eg) >= t.cert_a && rct2_cert<NDIM>(e, x, d, t.cert_rc)))
      return false;
  }
  return true;
}

// HCS reconstruction weights (Sec. 4.1, psi = 256/175):
//   G^ = psi G~ - (101/420)(G_i + G_{i+1}) + (1/105)(G_{i-1} + G_{i+2})
//        - (1/2100)(G_{i-2} + G_{i+3})
template <class R>
__device__ __forceinline__ R hcs(R gt, R gm2, R gm1, R g0, R gp1, R gp2, R gp3) {
  return R(256.0 / 175.0) * gt - R(101.0 / 420.0) * (g0 + gp1) + R(1.0 / 105.0) * (gm1 + gp2) -
         R(1.0 / 2100.0) * (gm2 + gp3);
}

// ---------------------------------------------------------------------------
// Shared-memory layout of one tile.
// ---------------------------------------------------------------------------
template <int NDIM, int DIR, class T>
struct Smem {
  static constexpr int NF = NDIM + 4;
  // per node: W (NF), velocity (NDIM), p, c, rho*ctilde^2, G (NF)
  static constexpr int NODE_DOUBLES = 2 * NF + NDIM + 3;
  // per midpoint: shared flux components (NF-1), alpha flux of G^- and G^+
  static constexpr int MID_DOUBLES = NF + 1;
  // + per node: whether it passes the limiters' threshold tests
  static constexpr size_t BYTES =
      sizeof(double) * (size_t)(NODE_DOUBLES * T::NN + MID_DOUBLES * T::NM) + sizeof(int) * (size_t)T::NN;
  double *W, *vel, *p, *c, *rct, *G, *F, *am, *ap;
  int *nok;
  __device__ Smem(double *base) {
    W = base;
    vel = W + NF * T::NN;
    p = vel + NDIM * T::NN;
    c = p + T::NN;
    rct = c + T::NN;
    G = rct + T::NN;
    F = G + NF * T::NN;
    am = F + (NF - 1) * T::NM;
    ap = am + T::NM;
    nok = (int *)(ap + T::NM);
  }
  // node slot of (line l, node s): consecutive threads get consecutive slots
  static __device__ __forceinline__ int nslot(int l, int s) {
    return DIR == 0 ? l * T::NS + s : s * T::TL + l;
  }
  static __device__ __forceinline__ int mslot(int l, int m) {
    return DIR == 0 ? l * T::TM + m : m * T::TL + l;
  }
};

// Geometry of one line of a tile: first cell index, stride along the swept
// axis, cells on the line, and whether the line exists.
struct Line {
  long long base;
  long long stride;
  long long face;  // position of the line on a face normal to it (lower axis fastest)
  int n;
  bool valid;
};

// Geometry policy of the handle's grid: block (x, y, z) = (tile along DIR,
// block of lines, third axis).  dt and lambda come from the device step
// control (Sec. 3.3 directional split).
template <int NDIM, int DIR, class T>
struct GridGeo {
  const SweepArgs &a;
  int tile0;
  __device__ GridGeo(const SweepArgs &a_) : a(a_), tile0(blockIdx.x * (T::TM - 1)) {}
  __device__ Line line(int l) const {
    Line r;
    const int nx = a.n[0], ny = a.n[1];
    if (DIR == 0) {
      int y = blockIdx.y * T::TL + l;
      r.valid = y < ny;
      y = min(y, ny - 1);
      r.face = (long long)blockIdx.z * ny + y;
      r.base = r.face * nx;
      r.stride = 1;
      r.n = nx;
    } else {
      int x = blockIdx.y * T::TL + l;
      r.valid = x < nx;
      x = min(x, nx - 1);
      r.face = (long long)blockIdx.z * nx + x;
      if (DIR == 1) {
        r.base = (long long)blockIdx.z * nx * ny + x;
        r.stride = nx;
        r.n = ny;
      } else {
        r.base = (long long)blockIdx.z * nx + x;
        r.stride = (long long)nx * ny;
        r.n = a.n[2];
      }
    }
    return r;
  }
  __device__ double dt() const { return a.ctl->dt; }
  __device__ double inv_dx() const { return a.inv_dx; }
  // lambda_d = dt / (dx_d sigma_d), sigma_d = tau_d / sum(tau),
  // tau = max(|u_d| + c)/dx_d of the stage input (Sec. 3.3).
  __device__ double lam() const {
    if (NDIM == 1) return a.ctl->dt * a.inv_dx;
    double tsum = 0.0;
#pragma unroll
    for (int j = 0; j < NDIM; ++j) tsum += __longlong_as_double(a.ctl->smax[a.stage][j]) * a.inv_dx_all[j];
    return a.ctl->dt * tsum / __longlong_as_double(a.ctl->smax[a.stage][DIR]);
  }
  __device__ unsigned long long *smax_slot(int j) const { return &a.ctl->smax[a.stage + 1][j]; }
  // mixed path: scaling of the L array (see SweepArgs::l_raw)
  __device__ double l_unit() const { return a.l_unit; }
  __device__ double accum_scale() const { return a.accum_scale; }
};

// ---------------------------------------------------------------------------
// The FP64 sweep body (the mixed-precision body is wcns_mixed_body.cuh).
// ---------------------------------------------------------------------------
template <int NDIM, int DIR, class R, class T, class Geo>
__device__ __forceinline__ void sweep_body(const SweepArgs &a, const Geo &geo, double *smem_raw) {
  static_assert(sizeof(R) == 8, "sweep_body is the FP64 body");
  using S = Smem<NDIM, DIR, T>;
  constexpr int NF = NDIM + 4, E = 2 + NDIM, A = 3 + NDIM;
  S sm(smem_raw);
  const int tid = threadIdx.x;
  const int tile0 = geo.tile0;  // first midpoint (= left face of cell tile0)
  const long long N = a.ncell;
  const EosConst eos = a.eos;

  // ---- 1+2: stage nodes and node work --------------------------------------
  for (int q = tid; q < T::NN; q += T::THREADS) {
    const int l = DIR == 0 ? q / T::NS : q % T::TL;
    const int s = DIR == 0 ? q % T::NS : q / T::TL;
    const Line ln = geo.line(l);
    const int n = ln.n;
    const int pos = tile0 - 3 + s;
    // no needed midpoint reads a node of a line beyond the grid or past the
    // line's last ghost layer (the last, partial tile of a line)
    if (!ln.valid || pos > n + 2) continue;
    double w[NF];
    bool dirichlet = false, flip = false;
    int src = pos;
    if (pos < -3 || pos > n + 2) {
      src = min(max(pos, 0), n - 1);  // outside every stencil: any valid cell
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
      const long long idx = ln.base + (long long)src * ln.stride;
#pragma unroll
      for (int f = 0; f < NF; ++f) w[f] = __ldg(a.W_in + (long long)f * N + idx);
      if (flip) w[2 + DIR] = -w[2 + DIR];
    }
    // Sec. 2, with Gamma = 1/(gbar-1) and Pi = gbar pbar/(gbar-1):
    //   p = (rho e - Pi)/Gamma,  pbar = Pi/(Gamma+1),
    //   rho c^2 = gbar (p + pbar) = ((Gamma+1) rho e - Pi)/Gamma^2,
    // with one division for 1/rho and one for 1/(Gamma (Gamma+1)).
    const double rho = w[0] + w[1];
    const double ir = div_nr(1.0, rho);
    double v[NDIM], m2 = 0.0;
#pragma unroll
    for (int j = 0; j < NDIM; ++j) {
      v[j] = w[2 + j] * ir;
      m2 = fma(w[2 + j], v[j], m2);
    }
    const double rhoe = w[E] - 0.5 * m2;
    const double Gam = mixGamma(eos, w[A]);
    const double Pi = mixPi(eos, w[A]);
    const double x = div_nr(1.0, Gam * (Gam + 1.0));
    const double iG = (Gam + 1.0) * x;
    const double p = (rhoe - Pi) * iG;
    const double c = sqrt(((Gam + 1.0) * rhoe - Pi) * (iG * iG) * ir);
    const double rct = rhoe - Pi * (Gam * x);
    const int slot = S::nslot(l, s);
#pragma unroll
    for (int f = 0; f < NF; ++f) sm.W[f * T::NN + slot] = w[f];
#pragma unroll
    for (int j = 0; j < NDIM; ++j) sm.vel[j * T::NN + slot] = v[j];
    sm.p[slot] = p;
    sm.c[slot] = c;
    sm.rct[slot] = rct;
    if (a.scheme == SCHEME_PP) sm.nok[slot] = state_passes<NDIM>(eos, a.tol, w);
    const double un = v[DIR];
    sm.G[0 * T::NN + slot] = w[0] * un;
    sm.G[1 * T::NN + slot] = w[1] * un;
#pragma unroll
    for (int j = 0; j < NDIM; ++j) sm.G[(2 + j) * T::NN + slot] = w[2 + j] * un + (j == DIR ? p : 0.0);
    sm.G[E * T::NN + slot] = (w[E] + p) * un;
    sm.G[A * T::NN + slot] = w[A] * un;
    // input admissibility (Sec. 2), counted once per interior cell
    if (DIR == 0 && ln.valid && s >= 3 && s < 3 + T::TM - 1 && pos < n) {
      const bool ok = w[0] >= 0.0 && w[1] >= 0.0 && w[A] >= 0.0 && w[A] <= 1.0 && rct > 0.0 &&
                      finite64(rhoe) && finite64(c);
      if (!ok) atomicAdd(&a.stats->inadmissible, 1ull);
    }
  }
  __syncthreads();

  const double dt = geo.dt();
  const double lam = geo.lam();
  const float l2f = (float)(2.0 * lam);  // for the flux-limiter certification
  const double eps4 = 4.0 * a.eps_is;  // IS epsilon for the indicators scaled by 4

  // ---- 3: midpoint fluxes ---------------------------------------------------
  int nlim_i = 0, nhard_i = 0, nlim_f = 0, nhard_f = 0, nslow = 0;
  for (int q = tid; q < T::NM; q += T::THREADS) {
    const int l = DIR == 0 ? q / T::TM : q % T::TL;
    const int m = DIR == 0 ? q % T::TM : q / T::TL;
    const int si = m + 2;  // node i; node i+1 is m + 3
    // Tiles overlap by one midpoint: count limiter events once per midpoint.
    const Line lnm = geo.line(l);
    // faces past the line's last face (partial tiles) and lines beyond the
    // grid are used by no updated cell
    if (!lnm.valid || tile0 + m > lnm.n) continue;
    const int cnt = (m < T::TM - 1 || tile0 + m == lnm.n) && tile0 + m <= lnm.n && lnm.valid;
    const int ni = S::nslot(l, si), ni1 = S::nslot(l, si + 1);
    double Wi[NF], Wi1[NF], vi[NDIM];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      Wi[f] = sm.W[f * T::NN + ni];
      Wi1[f] = sm.W[f * T::NN + ni1];
    }
#pragma unroll
    for (int j = 0; j < NDIM; ++j) vi[j] = sm.vel[j * T::NN + ni];
    const double pi_ = sm.p[ni];

    double vr[NDIM];  // velocity of node i+1
#pragma unroll
    for (int j = 0; j < NDIM; ++j) vr[j] = sm.vel[j * T::NN + ni1];
    // First-order HLLC flux from the nodes (Sec. 3.2), split into G^{HLLC,-}
    // and G^{HLLC,+}; in FP64 where it is used: the first-order scheme and
    // the flux limiter wherever its FP32 certification fails.
    auto first_order = [&](double *GHm, double *GHp) {
      double GH[NF], uH;
      hllc<NDIM, DIR, double>(Wi, vi, pi_, Wi[0] + Wi[1], sm.c[ni], Wi1, vr, sm.p[ni1], Wi1[0] + Wi1[1],
                              sm.c[ni1], GH, uH);
#pragma unroll
      for (int f = 0; f < NF; ++f) GHm[f] = GHp[f] = GH[f];
      GHm[A] = GH[A] - Wi[A] * uH;
      GHp[A] = GH[A] - Wi1[A] * uH;
    };

    double Gm[NF], Gp[NF];
    if (a.scheme == SCHEME_HLLC1) {
      first_order(Gm, Gp);
    } else {
      // Steps 1-2: primitive deviations from node i, projected with
      // Rinv_{i+1/2} (App. A; means of a1r1, a2r2, rho and c of nodes i, i+1).
      const double ar1 = 0.5 * (Wi[0] + Wi1[0]);
      const double ar2 = 0.5 * (Wi[1] + Wi1[1]);
      const double rb = ar1 + ar2;
      const double cb = 0.5 * (sm.c[ni] + sm.c[ni1]);
      const double irc = div_nr(1.0, rb * cb);
      const double ic = irc * rb;  // 1/c without another division
      const double k1 = ar1 * irc * ic, k2 = ar2 * irc * ic;
      double U[6][NF];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        double dv[NF];
        if (j == 2) {
#pragma unroll
          for (int f = 0; f < NF; ++f) dv[f] = 0.0;
        } else {
          const int sl = S::nslot(l, m + j);
          dv[0] = sm.W[0 * T::NN + sl] - Wi[0];
          dv[1] = sm.W[1 * T::NN + sl] - Wi[1];
#pragma unroll
          for (int k = 0; k < NDIM; ++k) dv[2 + k] = sm.vel[k * T::NN + sl] - vi[k];
          dv[E] = sm.p[sl] - pi_;
          dv[A] = sm.W[A * T::NN + sl] - Wi[A];
        }
        U[j][0] = dv[2 + DIR] - irc * dv[E];
        U[j][1] = dv[0] - k1 * dv[E];
        U[j][2] = dv[1] - k2 * dv[E];
        int row = 3;
#pragma unroll
        for (int k = 0; k < NDIM; ++k)
          if (k != DIR) U[j][row++] = dv[2 + k];
        U[j][NF - 2] = dv[A];
        U[j][NF - 1] = dv[2 + DIR] + irc * dv[E];
      }
      // Step 3: left/right WCNS-IS per characteristic field.
      double UL[NF], UR[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        UL[f] = wenois_c0_x4(U[0][f], U[1][f], U[3][f], U[4][f], eps4);
        UR[f] = wenois_p0_x4(U[5][f], U[4][f], U[3][f], U[1][f], eps4);
      }
      // Steps 4-5: back-project, add node i, V -> W.
      double WL[NF], WR[NF], VL[NF], VR[NF];  // V: (a1r1, a2r2, vel.., p, a1)
      const double h1 = 0.5 * ar1 * ic, h2 = 0.5 * ar2 * ic;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const double *Us = side ? UR : UL;
        double *V = side ? VR : VL;
        double *W = side ? WR : WL;
        const double dac = Us[NF - 1] - Us[0];
        V[0] = Wi[0] + (Us[1] + h1 * dac);
        V[1] = Wi[1] + (Us[2] + h2 * dac);
        int row = 3;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
          double dvk;
          if (k == DIR) {
            dvk = 0.5 * (Us[0] + Us[NF - 1]);
          } else {
            dvk = Us[row];
            ++row;
          }
          V[2 + k] = vi[k] + dvk;
        }
        V[E] = pi_ + 0.5 * rb * cb * dac;
        V[A] = Wi[A] + Us[NF - 2];
        const double rho = V[0] + V[1];
        double k2s = 0.0;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
          W[2 + k] = rho * V[2 + k];
          k2s = fma(V[2 + k], V[2 + k], k2s);
        }
        W[0] = V[0];
        W[1] = V[1];
        W[E] = fma(V[E], mixGamma(eos, V[A]), mixPi(eos, V[A])) + 0.5 * rho * k2s;
        W[A] = V[A];
      }
      // Interpolation limiter (Sec. 5.1): left toward W_i, right toward W_{i+1};
      // nothing to do where the node and the interpolated state pass every
      // threshold test (and the hard switch cannot fire after that).
      if (a.scheme == SCHEME_PP) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          double *W = side ? WR : WL;
          double *V = side ? VR : VL;
          if (a.tol.hs_implied && sm.nok[side ? ni1 : ni] && state_passes<NDIM>(eos, a.tol, W)) continue;
          nslow += cnt;
          const int fl = interp_limit<NDIM>(eos, a.tol, side ? Wi1 : Wi, W);
          nlim_i += cnt * (fl & 1);
          nhard_i += cnt * (fl >> 1);
          if (fl) {  // a limited state: primitives again from W
            const double r = W[0] + W[1];
            const double ir = 1.0 / r;
            double mm = 0.0;
#pragma unroll
            for (int k = 0; k < NDIM; ++k) {
              V[2 + k] = W[2 + k] * ir;
              mm = fma(W[2 + k], V[2 + k], mm);
            }
            V[0] = W[0];
            V[1] = W[1];
            V[E] = (W[E] - 0.5 * mm - mixPi(eos, W[A])) / mixGamma(eos, W[A]);
            V[A] = W[A];
          }
        }
      }
      // Step 6: midpoint HLLC; rho c^2 = ((Gamma+1) p + Pi)/Gamma (Sec. 2).
      double Gt[NF], ut, cs[2];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const double *V = side ? VR : VL;
        const double Gam = mixGamma(eos, V[A]);
        cs[side] = sqrt(div_nr((Gam + 1.0) * V[E] + mixPi(eos, V[A]), Gam * (V[0] + V[1])));
      }
      hllc<NDIM, DIR, double>(WL, VL + 2, VL[E], VL[0] + VL[1], cs[0], WR, VR + 2, VR[E], VR[0] + VR[1], cs[1],
                              Gt, ut);
      // Steps 7-8: HCS reconstruction from node fluxes and velocities.
      double Gh[NF];
      const int s0 = S::nslot(l, m), s1 = S::nslot(l, m + 1), s4 = S::nslot(l, m + 4), s5 = S::nslot(l, m + 5);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const double *g = sm.G + f * T::NN;
        Gh[f] = hcs<double>(Gt[f], g[s0], g[s1], g[ni], g[ni1], g[s4], g[s5]);
      }
      const double *un = sm.vel + DIR * T::NN;
      const double uh = hcs<double>(ut, un[s0], un[s1], un[ni], un[ni1], un[s4], un[s5]);
      // Step 9: G^-_{i+1/2} and G^+_{i+1/2}.
#pragma unroll
      for (int f = 0; f < NF; ++f) Gm[f] = Gp[f] = Gh[f];
      Gm[A] = Gh[A] - Wi[A] * uh;
      Gp[A] = Gh[A] - Wi1[A] * uh;
      // Flux limiter (Sec. 5.2), unless certified to leave the fluxes as they
      // are (the first-order flux then in FP32 with error bounds only).
      if (a.scheme == SCHEME_PP) {
        double Fi[NF], Fi1[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          Fi[f] = sm.G[f * T::NN + ni];
          Fi1[f] = sm.G[f * T::NN + ni1];
        }
        Fi[A] = 0.0;
        Fi1[A] = 0.0;
        float gH[NF + 1], eH[NF + 1];
        const bool cert =
            a.tol.hs_implied &&
            hllc1_bound32<NDIM, DIR>(Wi, vi, pi_, sm.c[ni], Wi1, vr, sm.p[ni1], sm.c[ni1], gH, eH) &&
            flux_certified<NDIM>(eos, a.tol, l2f, Wi, Wi1, Fi, Fi1, gH, eH, Gh, Gm[A], Gp[A]);
        if (!cert) {
          nslow += cnt;
          double GHm[NF], GHp[NF];
          first_order(GHm, GHp);
          const int fl = flux_limit<NDIM>(eos, a.tol, Wi, Wi1, Fi, Fi1, GHm, GHp, lam, Gm, Gp);
          nlim_f += cnt * (fl & 1);
          nhard_f += cnt * (fl >> 1);
        }
      }
    }
    const int ms = S::mslot(l, m);
#pragma unroll
    for (int f = 0; f < NF - 1; ++f) sm.F[f * T::NM + ms] = Gm[f];
    sm.am[ms] = Gm[A];
    sm.ap[ms] = Gp[A];
  }
  if (nlim_i) atomicAdd(&a.stats->interp_limited, (unsigned long long)nlim_i);
  if (nhard_i) atomicAdd(&a.stats->interp_hard, (unsigned long long)nhard_i);
  if (nlim_f) atomicAdd(&a.stats->flux_limited, (unsigned long long)nlim_f);
  if (nhard_f) atomicAdd(&a.stats->flux_hard, (unsigned long long)nhard_f);
  if (nslow) atomicAdd(&a.stats->fp64_fallbacks, (unsigned long long)nslow);
  __syncthreads();

  // ---- 4: cell update ------------------------------------------------------
  // Wave-speed maxima as bit patterns: |u_d| + c >= 0 (or NaN), and
  // non-negative doubles order like their bits, a NaN above every number.
  unsigned long long smax_local[NDIM];
#pragma unroll
  for (int j = 0; j < NDIM; ++j) smax_local[j] = 0ull;
  int midpoints_done = 0;
  const double idx_ = geo.inv_dx();
  const bool has_a = (__double_as_longlong(a.rk_a) << 1) != 0;  // a != 0, an integer test
  for (int q = tid; q < T::TL * (T::TM - 1); q += T::THREADS) {
    const int l = DIR == 0 ? q / (T::TM - 1) : q % T::TL;
    const int m = DIR == 0 ? q % (T::TM - 1) : q / T::TL;
    const Line ln = geo.line(l);
    const int pos = tile0 + m;
    if (!ln.valid || pos >= ln.n) continue;
    ++midpoints_done;
    const long long idx = ln.base + (long long)pos * ln.stride;
    const int ml = S::mslot(l, m), mr = S::mslot(l, m + 1);
    double upd[NF];
#pragma unroll
    for (int f = 0; f < NF - 1; ++f) upd[f] = (sm.F[f * T::NM + ml] - sm.F[f * T::NM + mr]) * idx_;
    upd[A] = (sm.ap[ml] - sm.am[mr]) * idx_;
    if (a.epilogue == EPI_WRITE) {
#pragma unroll
      for (int f = 0; f < NF; ++f) a.L[(long long)f * N + idx] = upd[f];
    } else if (a.epilogue == EPI_ACCUM) {
      // every load of the cell before its stores: the compiler cannot tell
      // the components apart, and would order each load after the last store
      double l0[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) l0[f] = a.L[(long long)f * N + idx];
#pragma unroll
      for (int f = 0; f < NF; ++f) a.L[(long long)f * N + idx] = l0[f] + upd[f];
    } else {
      const int ns = S::nslot(l, m + 3);
      double w[NF], lv[NF], wn[NF];
      bool finite = true;
      // loads first, as above (W_out may be any other array)
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        lv[f] = a.read_L ? a.L[(long long)f * N + idx] : 0.0;
        wn[f] = has_a ? a.Wn[(long long)f * N + idx] : 0.0;
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const double tot = a.read_L ? lv[f] + upd[f] : upd[f];
        w[f] = a.rk_a * wn[f] + a.rk_b * (sm.W[f * T::NN + ns] + dt * tot);
        finite = finite && finite64(w[f]);
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) a.W_out[(long long)f * N + idx] = w[f];
      if (!finite) atomicAdd(&a.stats->nonfinite, 1ull);
      // max(|u_d| + c) of the new state (Sec. 3.3) for the next stage:
      // c^2 = ((Gamma+1) rho e - Pi)/(Gamma^2 rho)
      const double rho = w[0] + w[1];
      const double ir = div_nr(1.0, rho);
      double m2 = 0.0;
#pragma unroll
      for (int j = 0; j < NDIM; ++j) m2 = fma(w[2 + j], w[2 + j], m2);
      const double rhoe = w[E] - 0.5 * m2 * ir;
      const double Gam = mixGamma(eos, w[A]);
      const double c = sqrt(div_nr((Gam + 1.0) * rhoe - mixPi(eos, w[A]), Gam * Gam * rho));
#pragma unroll
      for (int j = 0; j < NDIM; ++j) {
        const unsigned long long sj = (unsigned long long)__double_as_longlong(fabs(w[2 + j] * ir) + c);
        smax_local[j] = sj > smax_local[j] ? sj : smax_local[j];
      }
    }
  }
  if (a.epilogue == EPI_COMBINE) {
#pragma unroll
    for (int j = 0; j < NDIM; ++j) {
      unsigned long long b = smax_local[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, b, o);
        b = ob > b ? ob : b;
      }
      if ((tid & 31) == 0 && b) atomicMax(geo.smax_slot(j), b);
    }
  }
  // midpoint count (one per cell updated)
  for (int o = 16; o > 0; o >>= 1) midpoints_done += __shfl_xor_sync(0xffffffffu, midpoints_done, o);
  if ((tid & 31) == 0 && midpoints_done) atomicAdd(&a.stats->midpoints, (unsigned long long)midpoints_done);
}

// Resident blocks per SM the FP64 register allocation targets: two of 128
// threads (up to 255 registers each), else one.
template <int NDIM, int DIR, class R, class T>
__global__ void __launch_bounds__(T::THREADS, T::THREADS <= 128 ? 2 : 1) sweep_kernel(const SweepArgs a) {
  extern __shared__ double smem_raw[];
  if (!a.ctl->active) return;  // a finished advance: the step is a no-op
  sweep_body<NDIM, DIR, R, T>(a, GridGeo<NDIM, DIR, T>(a), smem_raw);
}

// Blocks of a sweep with tile T: (tiles along DIR, line blocks, third axis).
template <int DIR, class T>
dim3 sweep_grid(const SweepArgs &a) {
  dim3 grid((a.n[DIR] + T::TM - 2) / (T::TM - 1), 1, 1);
  if (DIR == 0) {
    grid.y = (a.n[1] + T::TL - 1) / T::TL;
    grid.z = a.n[2];
  } else {
    grid.y = (a.n[0] + T::TL - 1) / T::TL;
    grid.z = DIR == 1 ? a.n[2] : a.n[1];
  }
  return grid;
}

template <class T>
long long grid_blocks(const dim3 &g) {
  return (long long)g.x * g.y * g.z;
}

// Launch one sweep with tile T.
template <int NDIM, int DIR, class R, class T = Tile<NDIM, DIR>>
cudaError_t launch_sweep_t(const SweepArgs &a, cudaStream_t st) {
  const size_t bytes = Smem<NDIM, DIR, T>::BYTES;
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = configure_once(configured, [&] {
    return cudaFuncSetAttribute(sweep_kernel<NDIM, DIR, R, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
  });
  if (e != cudaSuccess) return e;
  sweep_kernel<NDIM, DIR, R, T><<<sweep_grid<DIR, T>(a), T::THREADS, bytes, st>>>(a);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_sweep_any(int ndim, int dir, const SweepArgs &a, cudaStream_t s) {
  switch (ndim * 4 + dir) {
    case 4: return launch_sweep_t<1, 0, R>(a, s);
    case 8: return launch_sweep_t<2, 0, R>(a, s);
    case 9: return launch_sweep_t<2, 1, R>(a, s);
    case 12: return launch_sweep_t<3, 0, R>(a, s);
    case 13: return launch_sweep_t<3, 1, R>(a, s);
    case 14: return launch_sweep_t<3, 2, R>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wcns
