// Mixed-precision instantiation of the directional sweep: characteristic
// projection, WCNS-IS interpolation and HLLC fluxes in FP32 (deviation
// form); node pressure, stored fluxes, limiter theta solves and state
// accumulation in FP64 (wcns_mixed_body.cuh).
#include "wcns_mixed_body.cuh"

namespace wcns {
cudaError_t launch_sweep_mixed(int ndim, int dir, const SweepArgs &a, cudaStream_t s) {
  switch (ndim * 4 + dir) {
    case 4: return launch_sweep_mixed_t<1, 0>(a, s);
    case 8: return launch_sweep_mixed_t<2, 0>(a, s);
    case 9: return launch_sweep_mixed_t<2, 1>(a, s);
    case 12: return launch_sweep_mixed_t<3, 0>(a, s);
    case 13: return launch_sweep_mixed_t<3, 1>(a, s);
    case 14: return launch_sweep_mixed_t<3, 2>(a, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace wcns
