// Tensor-core split product (placeholder until the tcgen05 kernels land).
#include "evd_ozaki.h"

namespace evd {

size_t ozaki_scratch_bytes(int64_t m, int64_t n, int64_t k, int slices) {
  (void)m; (void)n; (void)k; (void)slices;
  return 256;
}
bool ozaki_eligible(const Gemm& g) {
  (void)g;
  return false;
}
evd_status_t ozaki_gemm(const Gemm& g, int slices, void* scratch, size_t scratch_bytes, cudaStream_t s) {
  (void)g; (void)slices; (void)scratch; (void)scratch_bytes; (void)s;
  return EVD_ERR_NOT_SUPPORTED;
}

}  // namespace evd
