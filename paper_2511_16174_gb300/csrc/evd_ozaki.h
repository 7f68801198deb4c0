// Tensor-core split product: FP64 operands split into 7-bit bfloat16 slices
// (balanced base-128 digits after a per-row / per-column power-of-two scaling),
// slice pairs multiplied with tcgen05.mma kind::f16 into FP32 accumulators in
// tensor memory that stay exact integers, drained into 64-bit integer sums and
// converted to FP64 once per output element.
#pragma once

#include "evd_internal.h"

namespace evd {

size_t ozaki_scratch_bytes(int64_t m, int64_t n, int64_t k, int slices);

// A batch of equally shaped products C_p = alpha op(A_p) op(B_p) + beta C_p with
// A_p = A + p sA, B_p = B + p sB, C_p = C + p sC (element offsets, may be negative),
// in one split and one tensor-core launch.  Problem 0 may be truncated: its A view
// has only first_k K-elements (the rest read as zero) and it writes only first_m
// rows of C.  Needs K <= 512 when count > 1.
struct Batch {
  int count = 1;
  int64_t sA = 0, sB = 0, sC = 0;
  int64_t first_k = -1, first_m = -1;
};
size_t ozaki_scratch_bytes_batched(int64_t m, int64_t n, int64_t k, int slices, int count);
evd_status_t ozaki_gemm_batched(const Gemm& g, const Batch& bt, int slices, void* scratch, size_t scratch_bytes,
                                cudaStream_t s);
bool ozaki_eligible(const Gemm& g);
evd_status_t ozaki_gemm(const Gemm& g, int slices, void* scratch, size_t scratch_bytes, cudaStream_t s);

}  // namespace evd
