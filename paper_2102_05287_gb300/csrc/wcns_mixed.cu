// Mixed-precision instantiation of the directional sweep: characteristic
// projection, WCNS-IS interpolation and HLLC fluxes in FP32; node pressure
// and sound speed, limiter blending and state accumulation in FP64.
#include "wcns_sweep.cuh"

namespace wcns {
cudaError_t launch_sweep_mixed(int ndim, int dir, const SweepArgs &a, cudaStream_t s) {
  return launch_sweep_any<float>(ndim, dir, a, s);
}
}  // namespace wcns
