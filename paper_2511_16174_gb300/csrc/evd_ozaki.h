// Tensor-core split product: FP64 operands split into 7-bit bfloat16 slices
// (balanced base-128 digits after a per-row / per-column power-of-two scaling),
// slice pairs multiplied with tcgen05.mma kind::f16 into FP32 accumulators in
// tensor memory that stay exact integers, drained into 64-bit integer sums and
// converted to FP64 once per output element.
#pragma once

#include <cuda_bf16.h>

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
// The least scratch of one product (no K-split; the product lowers its split count to
// what the scratch holds).
size_t ozaki_scratch_bytes_min(int64_t m, int64_t n, int64_t k, int slices);
// Read and clear the status word of the stand-alone products (evd_dgemm).
evd_status_t standalone_status_take(int* code, int* info);
evd_status_t ozaki_gemm_batched(const Gemm& g, const Batch& bt, int slices, void* scratch, size_t scratch_bytes,
                                cudaStream_t s);
bool ozaki_eligible(const Gemm& g);
evd_status_t ozaki_gemm(const Gemm& g, int slices, void* scratch, size_t scratch_bytes, cudaStream_t s);

// An A operand split once and used by several products: the slices of a
// symmetric m x m matrix (lower triangle stored) in 128-row tiles, K padded to 32,
// with its per-row scales.  The double-blocked SBR's Z products of one block read
// principal submatrices of the same stale trailing matrix (Sec. 4.1).
struct SplitOperand {
  __nv_bfloat16* S = nullptr;
  int* e = nullptr;
  int64_t rows = 0, rows_pad = 0, K_pad = 0;
  int slices = 0;
  size_t bytes = 0;  // of the buffer it occupies
};
size_t ozaki_presplit_bytes(int64_t m, int slices);
evd_status_t ozaki_presplit_sym(const double* A, int64_t lda, int64_t m, int slices, void* buf, size_t bytes,
                                const char* tag, SplitOperand* out, cudaStream_t s);
// C = alpha A(off:, off:) op(B) + beta C with A the presplit operand (g.A ignored;
// g.m == g.k == rows - off, off a multiple of 16, g.ta == 'N').  The row scales
// are those of the whole operand's rows.  Scratch: ozaki_presplit_gemm_bytes.
size_t ozaki_presplit_gemm_bytes(int64_t m, int64_t n, int slices);
evd_status_t ozaki_gemm_presplit(const Gemm& g, const SplitOperand& sa, int64_t off, void* scratch,
                                 size_t scratch_bytes, cudaStream_t s);

}  // namespace evd
