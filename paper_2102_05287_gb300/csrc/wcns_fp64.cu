// FP64 instantiation of the directional sweep: every step of the RHS in FP64.
#include "../../include/wcns.h"
#include "wcns_sweep.cuh"

namespace wcns {
cudaError_t launch_sweep_fp64(int ndim, int dir, const SweepArgs &a, cudaStream_t s) {
  return launch_sweep_any<double>(ndim, dir, a, s);
}

namespace {
__global__ void division_check_kernel(const double *__restrict__ a, const double *__restrict__ b,
                                      double *__restrict__ q, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    q[i] = div_nr(a[i], b[i]);
}

// One case per thread: the sweeps' certification decision and the FP64
// limiter's outcome on the same inputs (row layouts as in wcns.h).
template <int NDIM>
__global__ void limiter_cert_check_kernel(int kind, const double *__restrict__ rows, long long n, EosConst eos,
                                          LimTol tol, int *__restrict__ cert, int *__restrict__ exact) {
  constexpr int NF = NDIM + 4, A = 3 + NDIM;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    auto same = [](const double *x, const double *y) {
      bool eq = true;
#pragma unroll
      for (int f = 0; f < NF; ++f) eq = eq && __double_as_longlong(x[f]) == __double_as_longlong(y[f]);
      return eq;
    };
    if (kind == 0) {
      const double *r = rows + i * (2 * NF);
      double Wn[NF], Wt[NF], W0[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        Wn[f] = r[f];
        Wt[f] = W0[f] = r[NF + f];
      }
      cert[i] = tol.hs_implied && state_passes<NDIM>(eos, tol, Wn) && state_passes<NDIM>(eos, tol, Wt);
      const int fl = interp_limit<NDIM>(eos, tol, Wn, Wt);
      exact[i] = fl == 0 && same(Wt, W0);
    } else if (kind == 1) {
      const double *r = rows + i * (8 * NF + 1);
      double Wi[NF], Wi1[NF], Fi[NF], Fi1[NF], GHm[NF], GHp[NF], Gm[NF], Gp[NF], Gm0[NF], Gp0[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        Wi[f] = r[f];
        Wi1[f] = r[NF + f];
        Fi[f] = r[2 * NF + f];
        Fi1[f] = r[3 * NF + f];
        GHm[f] = r[4 * NF + f];
        GHp[f] = f == A ? r[5 * NF + f] : GHm[f];
        Gm[f] = Gm0[f] = r[6 * NF + f];
        Gp[f] = Gp0[f] = f == A ? r[7 * NF + f] : Gm[f];
      }
      Fi[A] = 0.0;
      Fi1[A] = 0.0;
      const double lam = r[8 * NF];
      const float l2f = (float)(2.0 * lam);
      // the given first-order flux, known to within its truncation
      float gH[NF + 1], eH[NF + 1];
#pragma unroll
      for (int f = 0; f <= NF; ++f) {
        gH[f] = trunc32(f < A ? GHm[f] : f == A ? GHm[A] : GHp[A]);
        eH[f] = 1.9073486328125e-06f * fabsf(gH[f]) + CTINY;
      }
      cert[i] = tol.hs_implied && flux_certified<NDIM>(eos, tol, l2f, Wi, Wi1, Fi, Fi1, gH, eH, Gm, Gm[A], Gp[A]);
      const int fl = flux_limit<NDIM>(eos, tol, Wi, Wi1, Fi, Fi1, GHm, GHp, lam, Gm, Gp);
      exact[i] = fl == 0 && same(Gm, Gm0) && same(Gp, Gp0);
    } else {
      // nodes i, i+1 (W, velocity, p, c), node fluxes, high-order flux, lambda
      constexpr int NODE = NF + NDIM + 2;
      const double *r = rows + i * (2 * NODE + 3 * NF + 3);
      double Wi[NF], Wi1[NF], vi[NDIM], vr[NDIM], Fi[NF], Fi1[NF], Gm[NF], Gp[NF], Gm0[NF], Gp0[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        Wi[f] = r[f];
        Wi1[f] = r[NODE + f];
        Fi[f] = r[2 * NODE + f];
        Fi1[f] = r[2 * NODE + NF + f];
        Gm[f] = Gp[f] = Gm0[f] = Gp0[f] = r[2 * NODE + 2 * NF + f];
      }
#pragma unroll
      for (int j = 0; j < NDIM; ++j) {
        vi[j] = r[NF + j];
        vr[j] = r[NODE + NF + j];
      }
      const double pi = r[NF + NDIM], ci = r[NF + NDIM + 1];
      const double pr = r[NODE + NF + NDIM], cr = r[NODE + NF + NDIM + 1];
      Gm[A] = Gm0[A] = r[2 * NODE + 3 * NF];
      Gp[A] = Gp0[A] = r[2 * NODE + 3 * NF + 1];
      const double lam = r[2 * NODE + 3 * NF + 2];
      Fi[A] = 0.0;
      Fi1[A] = 0.0;
      const float l2f = (float)(2.0 * lam);
      // the sweeps' two routes: the bounded FP32 first-order flux with the
      // certification, and the FP64 flux with the FP64 limiter
      float gH[NF + 1], eH[NF + 1];
      cert[i] = tol.hs_implied &&
                hllc1_bound32<NDIM, NDIM - 1>(Wi, vi, pi, ci, Wi1, vr, pr, cr, gH, eH) &&
                flux_certified<NDIM>(eos, tol, l2f, Wi, Wi1, Fi, Fi1, gH, eH, Gm, Gm[A], Gp[A]);
      double GH[NF], uH, GHm[NF], GHp[NF];
      hllc<NDIM, NDIM - 1, double>(Wi, vi, pi, Wi[0] + Wi[1], ci, Wi1, vr, pr, Wi1[0] + Wi1[1], cr, GH, uH);
#pragma unroll
      for (int f = 0; f < NF; ++f) GHm[f] = GHp[f] = GH[f];
      GHm[A] = GH[A] - Wi[A] * uH;
      GHp[A] = GH[A] - Wi1[A] * uH;
      const int fl = flux_limit<NDIM>(eos, tol, Wi, Wi1, Fi, Fi1, GHm, GHp, lam, Gm, Gp);
      exact[i] = fl == 0 && same(Gm, Gm0) && same(Gp, Gp0);
    }
  }
}
}  // namespace
}  // namespace wcns

extern "C" int wcns_check_limiter_cert(int ndim, int kind, const double *rows, long long n, double eps_ar,
                                       double eps_a, double eps_rc, double gamma_g, double gamma_l, double pinf_l,
                                       int *cert, int *exact, void *stream) {
  if (ndim < 1 || ndim > 3 || kind < 0 || kind > 2 || n < 0 || (n > 0 && (!rows || !cert || !exact)))
    return WCNS_E_INVALID_ARG;
  if (!(gamma_g > 1.0) || !(gamma_l > 1.0) || !(pinf_l >= 0.0) || !(gamma_g <= gamma_l) || !isfinite(gamma_g) ||
      !isfinite(gamma_l) || !isfinite(pinf_l))
    return WCNS_E_INVALID_ARG;
  const double eps[3] = {eps_ar, eps_a, eps_rc};
  for (double x : eps)
    if (!(x >= 0.0) || !(x < 1e300)) return WCNS_E_INVALID_ARG;
  if (n == 0) return WCNS_OK;
  wcns::LimTol tol;
  tol.eps_ar = tol.hs_ar = eps_ar;
  tol.eps_a = tol.hs_a = eps_a;
  tol.eps_rc = tol.hs_rc = eps_rc;
  wcns::set_cert(tol);
  const wcns::EosConst eos = wcns::make_eos(gamma_g, gamma_l, pinf_l);
  const long long blocks = (n + 127) / 128 < 152 * 8 ? (n + 127) / 128 : 152 * 8;
  cudaStream_t st = (cudaStream_t)stream;
  switch (ndim) {
    case 1: wcns::limiter_cert_check_kernel<1><<<(int)blocks, 128, 0, st>>>(kind, rows, n, eos, tol, cert, exact); break;
    case 2: wcns::limiter_cert_check_kernel<2><<<(int)blocks, 128, 0, st>>>(kind, rows, n, eos, tol, cert, exact); break;
    default: wcns::limiter_cert_check_kernel<3><<<(int)blocks, 128, 0, st>>>(kind, rows, n, eos, tol, cert, exact); break;
  }
  return cudaGetLastError() == cudaSuccess ? WCNS_OK : WCNS_E_CUDA;
}

extern "C" int wcns_check_division(const double *a, const double *b, double *q, long long n, void *stream) {
  if (n < 0 || (n > 0 && (!a || !b || !q))) return WCNS_E_INVALID_ARG;
  if (n == 0) return WCNS_OK;
  const long long blocks = (n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8;
  wcns::division_check_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(a, b, q, n);
  return cudaGetLastError() == cudaSuccess ? WCNS_OK : WCNS_E_CUDA;
}
