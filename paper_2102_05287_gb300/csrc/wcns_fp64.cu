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
}  // namespace
}  // namespace wcns

extern "C" int wcns_check_division(const double *a, const double *b, double *q, long long n, void *stream) {
  if (n < 0 || (n > 0 && (!a || !b || !q))) return WCNS_E_INVALID_ARG;
  if (n == 0) return WCNS_OK;
  const long long blocks = (n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8;
  wcns::division_check_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(a, b, q, n);
  return cudaGetLastError() == cudaSuccess ? WCNS_OK : WCNS_E_CUDA;
}
