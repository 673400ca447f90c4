// Derivative-loss rows of the ipm equation: the instantiations of the kernel in
// djet_impl.cuh for this equation (one translation unit per equation, compiled in parallel).
#include "djet_impl.cuh"

namespace gn {
cudaError_t launch_djet_ipm(const JetArgs& a, int ord, cudaStream_t st, int64_t* warps_used) {
  return djet::launch_eq<GN_IPM>(a, ord, st, warps_used);
}
}  // namespace gn
