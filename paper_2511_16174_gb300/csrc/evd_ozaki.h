// Tensor-core split product: FP64 operands split into 7-bit bfloat16 slices
// (balanced base-128 digits after a per-row / per-column power-of-two scaling),
// slice pairs multiplied with tcgen05.mma kind::f16 into FP32 accumulators in
// tensor memory that stay exact integers, drained into 64-bit integer sums and
// converted to FP64 once per output element.
#pragma once

#include "evd_internal.h"

namespace evd {

size_t ozaki_scratch_bytes(int64_t m, int64_t n, int64_t k, int slices);
bool ozaki_eligible(const Gemm& g);
evd_status_t ozaki_gemm(const Gemm& g, int slices, void* scratch, size_t scratch_bytes, cudaStream_t s);

}  // namespace evd
