// Split-precision (Ozaki) Gram product on the tcgen05 tensor cores.
#include "gn_internal.cuh"

namespace gn {

int split_gram(gn_handle* h, const double* J, int64_t ld, int64_t nrows, double* G, int accumulate) {
  (void)h; (void)J; (void)ld; (void)nrows; (void)G; (void)accumulate;
  return GN_ERR_UNSUPPORTED;
}

}  // namespace gn
