// Ogita-Aishima eigenpair refinement (Ogita & Aishima, JJIAM 35, 2018), one or
// more steps, with FP64-accurate residual products:
//   R = I - X^T X,  S = X^T A X  (both symmetric by definition: only their lower
//                                 triangles are computed, then mirrored),
//   lam_i = s_ii / (1 - r_ii),
//   delta = 2 (||S - diag(lam)|| + ||A|| ||R||)       (Frobenius norms, which bound
//                                                      the 2-norms from above),
//           held at its largest value over the steps of one call,
//   E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i)  if |lam_i - lam_j| > delta
//        = r_ij / 2                                otherwise
//   X <- X + X E.
// Why delta never shrinks: X'^T X' - I = E^T E + ... to second order, and a pair
// that an earlier step left in the r_ij / 2 branch keeps its mixing, so a smaller
// delta in a later step would rotate it by E_ij ~ s_ij / (lam_j - lam_i), up to
// s_ij / delta, and leave an orthogonality error of that size squared.  Holding
// delta keeps every step's E within what the first step's delta allowed.
// X E needs only a few slices: E is at the error level of X, so a relative error of
// 2^-27 in the product (4 slices) is far below FP64 rounding of X.
#include <algorithm>
#include <cstdio>

#include "device_util.cuh"
#include "evd_internal.h"

namespace evd {

namespace {

// sum of squares of an m x n block (lower-only: i >= j, doubling the strict part
// when sym) into out[0] via per-CTA partials then one atomic per CTA is not
// deterministic; use a two-pass deterministic reduction instead.
__global__ void k_sumsq_partial(const double* A, int64_t lda, int64_t n, int mode, const double* lam, double* part) {
  // mode 0: plain sum of squares of the n x n matrix
  // mode 1: symmetric from lower triangle (off-diagonal counted twice)
  // mode 2: ||S - diag(lam)||^2
  __shared__ double red[256];
  const int64_t j = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double x;
    if (mode == 1) {
      if (i < j) continue;
      x = A[i + j * lda];
      s += (i == j) ? x * x : 2.0 * x * x;
      continue;
    }
    x = A[i + j * lda];
    if (mode == 2 && i == j) x -= lam[i];
    s += x * x;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[j] = red[0];
}

__global__ void k_sum_final(const double* part, int64_t n, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_add_identity(double* R, int64_t ldr, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) R[i + i * ldr] += 1.0;
}

// R and S are symmetric by definition and only their lower triangles are
// computed: mirror them into the upper triangles (a rounding asymmetry of S would
// otherwise enter E_ij + E_ji divided by the eigenvalue gap).  One thread per
// pair (i > j) of column j.
__global__ void k_mirror_lower2(double* R, double* S, int64_t ld, int64_t n) {
  const int64_t j = blockIdx.y;
  for (int64_t i = j + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    R[j + i * ld] = R[i + j * ld];
    S[j + i * ld] = S[i + j * ld];
  }
}

// norms[3] = max(norms[3], 2 (||S - diag|| + ||A|| ||R||)): the step's threshold,
// never below an earlier step's.
__global__ void k_delta(double* norms) {
  const double d = 2.0 * (sqrt(norms[2]) + sqrt(norms[0]) * sqrt(norms[1]));
  norms[3] = fmax(norms[3], d);
}

__global__ void k_lambda(const double* S, const double* R, int64_t ld, int64_t n, double* lam) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) lam[i] = S[i + i * ld] / (1.0 - R[i + i * ld]);
}

// E overwrites S.  norms[3] = delta (k_delta).
__global__ void k_form_E(double* S, const double* R, int64_t ld, int64_t n, const double* lam, const double* norms) {
  const int64_t j = blockIdx.y;
  const double delta = norms[3];
  const double lj = lam[j];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double li = lam[i];
    const double r = R[i + j * ld];
    double e;
    if (fabs(li - lj) > delta) e = (S[i + j * ld] + lj * r) / (lj - li);
    else e = 0.5 * r;
    S[i + j * ld] = e;
  }
}

__global__ void k_axpy_mat(const double* Y, int64_t ldy, double* X, int64_t ldx, int64_t n) {
  const int64_t j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    X[i + j * ldx] += Y[i + j * ldy];
}

}  // namespace

evd_status_t refine_run(const PlanCore& pc, const double* A0, int64_t lda0, double* w, double* Q, int64_t ldq,
                        int iters, const RefineWork& rw) {
  const int64_t n = pc.n;
  cudaStream_t s = pc.stream;
  if (n == 0) return EVD_OK;
  if (n > 65535) {
    // column-parallel helper kernels use grid.y = n
    return EVD_ERR_NOT_SUPPORTED;
  }
  double* norms = rw.vec + 2 * n;  // [0] ||A||^2, [1] ||R||^2, [2] ||S - diag||^2, [3] delta
  double* part = rw.vec + n;       // n partials
  double* lam = rw.vec;
  const unsigned rx = (unsigned)std::min<int64_t>(ceil_div(n, 256), 16);
  k_sumsq_partial<<<(unsigned)n, 256, 0, s>>>(A0, lda0, n, 1, nullptr, part); count_launch();
  k_sum_final<<<1, 256, 0, s>>>(part, n, norms + 0); count_launch();
  EVD_CUDA_TRY(cudaMemsetAsync(norms + 3, 0, sizeof(double), s));
  EVD_CUDA_TRY(cudaGetLastError());
  for (int it = 0; it < iters; ++it) {
    // R = I - X^T X (lower triangle)
    Gemm g1;
    g1.status = pc.status; g1.tag = "refine"; g1.lower = true;
    g1.ta = 'T'; g1.m = n; g1.n = n; g1.k = n; g1.A = Q; g1.lda = ldq; g1.B = Q; g1.ldb = ldq;
    g1.C = rw.R; g1.ldc = n; g1.alpha = -1.0; g1.beta = 0.0;
    evd_status_t st = gemm(g1, pc.ref_slices, rw.gemm_ws, rw.gemm_ws_bytes, s);
    if (st != EVD_OK) return st;
    k_add_identity<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(rw.R, n, n); count_launch();
    // AX = A0 X (A0 symmetric, lower stored)
    Gemm g2;
    g2.status = pc.status; g2.tag = "refine";
    g2.m = n; g2.n = n; g2.k = n; g2.A = A0; g2.lda = lda0; g2.a_sym_lower = true; g2.B = Q; g2.ldb = ldq;
    g2.C = rw.AX; g2.ldc = n; g2.alpha = 1.0; g2.beta = 0.0;
    st = gemm(g2, pc.ref_slices, rw.gemm_ws, rw.gemm_ws_bytes, s);
    if (st != EVD_OK) return st;
    // S = X^T AX (lower triangle)
    Gemm g3;
    g3.status = pc.status; g3.tag = "refine"; g3.lower = true;
    g3.ta = 'T'; g3.m = n; g3.n = n; g3.k = n; g3.A = Q; g3.lda = ldq; g3.B = rw.AX; g3.ldb = n;
    g3.C = rw.S; g3.ldc = n; g3.alpha = 1.0; g3.beta = 0.0;
    st = gemm(g3, pc.ref_slices, rw.gemm_ws, rw.gemm_ws_bytes, s);
    if (st != EVD_OK) return st;
    k_mirror_lower2<<<dim3(rx, (unsigned)n), 256, 0, s>>>(rw.R, rw.S, n, n); count_launch();
    k_lambda<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(rw.S, rw.R, n, n, lam); count_launch();
    k_sumsq_partial<<<(unsigned)n, 256, 0, s>>>(rw.R, n, n, 0, nullptr, part); count_launch();
    k_sum_final<<<1, 256, 0, s>>>(part, n, norms + 1); count_launch();
    k_sumsq_partial<<<(unsigned)n, 256, 0, s>>>(rw.S, n, n, 2, lam, part); count_launch();
    k_sum_final<<<1, 256, 0, s>>>(part, n, norms + 2); count_launch();
    k_delta<<<1, 1, 0, s>>>(norms); count_launch();
    k_form_E<<<dim3(rx, (unsigned)n), 256, 0, s>>>(rw.S, rw.R, n, n, lam, norms); count_launch();
    EVD_CUDA_TRY(cudaGetLastError());
    // X <- X + X E   (product into AX with few slices, then add)
    Gemm g4;
    g4.status = pc.status; g4.tag = "refine_xe";
    g4.m = n; g4.n = n; g4.k = n; g4.A = Q; g4.lda = ldq; g4.B = rw.S; g4.ldb = n;
    g4.C = rw.AX; g4.ldc = n; g4.alpha = 1.0; g4.beta = 0.0;
    st = gemm(g4, pc.xe_slices, rw.gemm_ws, rw.gemm_ws_bytes, s);
    if (st != EVD_OK) return st;
    k_axpy_mat<<<dim3(rx, (unsigned)n), 256, 0, s>>>(rw.AX, n, Q, ldq, n); count_launch();
    EVD_CUDA_TRY(cudaGetLastError());
  }
  EVD_CUDA_TRY(cudaMemcpyAsync(w, lam, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  return EVD_OK;
}

}  // namespace evd
