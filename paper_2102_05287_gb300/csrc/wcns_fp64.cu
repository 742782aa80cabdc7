// FP64 instantiation of the directional sweep: every step of the RHS in FP64.
#include "wcns_sweep.cuh"

namespace wcns {
cudaError_t launch_sweep_fp64(int ndim, int dir, const SweepArgs &a, cudaStream_t s) {
  return launch_sweep_any<double>(ndim, dir, a, s);
}
}  // namespace wcns
