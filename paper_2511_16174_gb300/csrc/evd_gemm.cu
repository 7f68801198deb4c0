// Dense products C = alpha op(A) op(B) + beta C in FP64.
//
// Two engines:
//  * a plain FP64 CUDA-core kernel (slices == 0), used for small or thin shapes;
//  * the tensor-core split product (slices 1..8, evd_ozaki.cu), used for the large
//    contractions of SBR (Eq. 1), the back transformation and the D&C merges.
#include <algorithm>
#include <cstdio>

#include "device_util.cuh"
#include "evd_internal.h"
#include "evd_ozaki.h"

namespace evd {

namespace {

// 32 x 64 tiles of 128 threads (4 x 4 per thread): at 58 registers a CTA takes 7.4K
// registers, so it fits on an SM beside a fused BC-Back wave CTA (which leaves 10K),
// and the D&C merges that run during the back transformation use the FP64 pipe the
// waves leave idle instead of waiting for whole SMs.
constexpr int BM = 32, BN = 64, BK = 16, NT = 128;

__device__ __forceinline__ double load_a(const Gemm& g, int64_t r, int64_t c) {
  // op(A)(r, c), 0 <= r < m, 0 <= c < k
  if (g.a_sym_lower) return (r >= c) ? g.A[r + c * g.lda] : g.A[c + r * g.lda];
  return (g.ta == 'N') ? g.A[r + c * g.lda] : g.A[c + r * g.lda];
}
__device__ __forceinline__ double load_b(const Gemm& g, int64_t r, int64_t c) {
  // op(B)(r, c), 0 <= r < k, 0 <= c < n
  return (g.tb == 'N') ? g.B[r + c * g.ldb] : g.B[c + r * g.ldb];
}

__device__ __forceinline__ void dgemm_tile(const Gemm& g, int64_t m0, int64_t n0);

__global__ void __launch_bounds__(NT) k_dgemm_simt(const Gemm g) {
  dgemm_tile(g, (int64_t)blockIdx.x * BM, (int64_t)blockIdx.y * BN);
}

// Many independent products in one launch: problem blockIdx.z, its tiles inside the
// grid of the largest one (the other CTAs leave at once).
__global__ void __launch_bounds__(NT) k_dgemm_simt_batched(const Gemm* __restrict__ gs) {
  const Gemm& g = gs[blockIdx.z];
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  if (m0 >= g.m || n0 >= g.n) return;
  dgemm_tile(g, m0, n0);
}

__device__ __forceinline__ void dgemm_tile(const Gemm& g, int64_t m0, int64_t n0) {
  if (g.lower && n0 > m0 + BM - 1) return;  // tile strictly above the diagonal
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int64_t k0 = 0; k0 < g.k; k0 += BK) {
    // A tile: 64 x 16
    for (int t = threadIdx.x; t < BM * BK; t += NT) {
      int i, kk;
      if (g.ta == 'N' || g.a_sym_lower) { i = t % BM; kk = t / BM; }
      else { kk = t % BK; i = t / BK; }
      int64_t r = m0 + i, c = k0 + kk;
      As[kk][i] = (r < g.m && c < g.k) ? load_a(g, r, c) : 0.0;
    }
    for (int t = threadIdx.x; t < BN * BK; t += NT) {
      int j, kk;
      if (g.tb == 'N') { kk = t % BK; j = t / BK; }
      else { j = t % BN; kk = t / BN; }
      int64_t r = k0 + kk, c = n0 + j;
      Bs[kk][j] = (r < g.k && c < g.n) ? load_b(g, r, c) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 8 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t r = m0 + tx + 8 * i, c = n0 + ty + 16 * j;
      if (r < g.m && c < g.n && (!g.lower || r >= c)) {
        double* p = g.C + r + c * g.ldc;
        double v = g.alpha * acc[i][j];
        if (g.beta != 0.0) v = fma(g.beta, *p, v);
        *p = v;
      }
    }
}

__global__ void k_scale(double* C, int64_t ldc, int64_t m, int64_t n, double beta, bool lower) {
  int64_t j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (lower && i < j) continue;
    double* p = C + i + j * ldc;
    *p = (beta == 0.0) ? 0.0 : beta * *p;
  }
}

// C (m x n, both <= 128) = alpha A^T B + beta C with a long K: partial products over
// K chunks of 256 rows in FP64 (one CTA per chunk), then a fixed-order sum.
constexpr int SK_CHUNK = 256;
__global__ void __launch_bounds__(256) k_atb_partial(const double* __restrict__ A, int64_t lda,
                                                     const double* __restrict__ B, int64_t ldb, int64_t m, int64_t n,
                                                     int64_t k, double* part) {
  __shared__ double As[32][129];
  __shared__ double Bs[32][129];
  const int64_t k0 = (int64_t)blockIdx.x * SK_CHUNK;
  const int tid = threadIdx.x;
  double acc[64];
  const int nout = (int)(m * n);
  for (int q = 0; q < 64; ++q) acc[q] = 0.0;
  for (int64_t kk = k0; kk < k0 + SK_CHUNK && kk < k; kk += 32) {
    __syncthreads();
    for (int idx = tid; idx < 32 * 128; idx += 256) {
      const int r = idx % 32, c = idx / 32;
      const int64_t K = kk + r;
      As[r][c] = (K < k && c < m) ? A[K + c * lda] : 0.0;
      Bs[r][c] = (K < k && c < n) ? B[K + c * ldb] : 0.0;
    }
    __syncthreads();
    for (int q = 0; q < 64; ++q) {
      const int o = tid + q * 256;
      if (o >= nout) break;
      const int i = o % (int)m, j = o / (int)m;
      double sacc = acc[q];
      for (int r = 0; r < 32; ++r) sacc = fma(As[r][i], Bs[r][j], sacc);
      acc[q] = sacc;
    }
  }
  for (int q = 0; q < 64; ++q) {
    const int o = tid + q * 256;
    if (o >= nout) break;
    part[(size_t)blockIdx.x * nout + o] = acc[q];
  }
}

__global__ void k_atb_sum(const double* part, int nchunks, int64_t m, int64_t n, double alpha, double beta, double* C,
                          int64_t ldc) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= m * n) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * m * n + o];
  const int64_t i = o % m, j = o / m;
  double* p = C + i + j * ldc;
  double v = alpha * s;
  if (beta != 0.0) v = fma(beta, *p, v);
  *p = v;
}

}  // namespace

evd_status_t gemm_simt_batched(const Gemm* host, int count, Gemm* dev, const char* tag, cudaStream_t s) {
  if (count <= 0) return EVD_OK;
  int64_t mt = 0, nt = 0;
  double flops = 0.0;
  for (int i = 0; i < count; ++i) {
    if (host[i].k <= 0 || host[i].lower || host[i].a_sym_lower) return EVD_ERR_INVALID_ARG;
    mt = std::max<int64_t>(mt, ceil_div(host[i].m, BM));
    nt = std::max<int64_t>(nt, ceil_div(host[i].n, BN));
    flops += 2.0 * (double)host[i].m * (double)host[i].n * (double)host[i].k;
  }
  if (nt > 65535 || count > 65535) return EVD_ERR_INVALID_ARG;
  EVD_CUDA_TRY(cudaMemcpyAsync(dev, host, sizeof(Gemm) * count, cudaMemcpyHostToDevice, s));
  StatScope sc(tag, s, flops, 0.0, "fp64_simt");
  k_dgemm_simt_batched<<<dim3((unsigned)mt, (unsigned)nt, (unsigned)count), NT, 0, s>>>(dev); count_launch();
  EVD_CUDA_TRY(cudaGetLastError());
  return EVD_OK;
}

size_t gemm_scratch_bytes(int64_t m, int64_t n, int64_t k, int slices) {
  if (slices <= 0) return 0;
  return ozaki_scratch_bytes(m, n, k, slices);
}

evd_status_t gemm(const Gemm& g, int slices, void* scratch, size_t scratch_bytes, cudaStream_t s) {
  if (g.m <= 0 || g.n <= 0) return EVD_OK;
  if (g.k <= 0 || g.alpha == 0.0) {
    if (g.beta == 1.0) return EVD_OK;
    for (int64_t j0 = 0; j0 < g.n; j0 += 65535) {
      int64_t cols = g.n - j0 < 65535 ? g.n - j0 : 65535;
      k_scale<<<dim3(4, (unsigned)cols), 256, 0, s>>>(g.C + j0 * g.ldc, g.ldc, g.m, cols, g.beta, false); count_launch();
    }
    EVD_CUDA_TRY(cudaGetLastError());
    return EVD_OK;
  }
  if (slices > 0 && (g.force_tc || ozaki_eligible(g))) return ozaki_gemm(g, slices, scratch, scratch_bytes, s);
  // small A^T B with a long K: split K across CTAs
  if (g.ta == 'T' && g.tb == 'N' && !g.lower && !g.a_sym_lower && g.m <= 128 && g.n <= 128 && g.m * g.n <= 64 * 256 &&
      g.k >= 4 * SK_CHUNK && scratch) {
    const int nch = (int)ceil_div(g.k, SK_CHUNK);
    if (scratch_bytes >= (size_t)nch * g.m * g.n * sizeof(double)) {
      StatScope sc(g.tag ? g.tag : "gemm", s, 2.0 * (double)g.m * (double)g.n * (double)g.k, 0.0, "fp64_splitk");
      double* part = static_cast<double*>(scratch);
      k_atb_partial<<<nch, 256, 0, s>>>(g.A, g.lda, g.B, g.ldb, g.m, g.n, g.k, part); count_launch();
      k_atb_sum<<<(unsigned)ceil_div(g.m * g.n, 256), 256, 0, s>>>(part, nch, g.m, g.n, g.alpha, g.beta, g.C, g.ldc); count_launch();
      EVD_CUDA_TRY(cudaGetLastError());
      return EVD_OK;
    }
  }
  dim3 grid((unsigned)ceil_div(g.m, BM), (unsigned)ceil_div(g.n, BN));
  if (grid.y > 65535) return EVD_ERR_INVALID_ARG;
  const double flops = (g.lower ? 1.0 : 2.0) * (double)g.m * (double)g.n * (double)g.k;
  StatScope sc(g.tag ? g.tag : "gemm", s, flops, 0.0, "fp64_simt");
  k_dgemm_simt<<<grid, NT, 0, s>>>(g); count_launch();
  EVD_CUDA_TRY(cudaGetLastError());
  return EVD_OK;
}

}  // namespace evd
