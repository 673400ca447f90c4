// Dispatch of the derivative-loss rows (the kernel is in djet_impl.cuh, instantiated per
// equation in djet_<equation>.cu).
#include "gn_internal.cuh"

namespace gn {

cudaError_t launch_djet_burgers(const JetArgs& a, int ord, cudaStream_t st, int64_t* warps_used);
cudaError_t launch_djet_ccf(const JetArgs& a, int ord, cudaStream_t st, int64_t* warps_used);
cudaError_t launch_djet_ipm(const JetArgs& a, int ord, cudaStream_t st, int64_t* warps_used);
cudaError_t launch_djet_boussinesq(const JetArgs& a, int ord, cudaStream_t st, int64_t* warps_used);

cudaError_t launch_djet(const JetArgs& a, int ord, cudaStream_t st, int64_t* warps_used) {
  if (ord != 1 && ord != 2) return cudaErrorInvalidValue;
  switch (a.eq) {
    case GN_BURGERS: return launch_djet_burgers(a, ord, st, warps_used);
    case GN_CCF: return launch_djet_ccf(a, ord, st, warps_used);
    case GN_IPM: return launch_djet_ipm(a, ord, st, warps_used);
    case GN_BOUSSINESQ: return launch_djet_boussinesq(a, ord, st, warps_used);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gn
