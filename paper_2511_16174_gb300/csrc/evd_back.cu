// Back transformation (Sec. 2.1.2), conventional order: X = Q_d, then
//   BC-Back:  X <- Q_b X   with Q_b the product of the bulge-chasing reflectors
//   SBR-Back: X <- Q_s X   with Q_s = prod_p (I - V_p T_p V_p^T)
//
// BC-Back ordering.  Q_b = H_{0,0} H_{0,1} ... H_{1,0} ... (sweep by sweep, step by
// step).  H_{j,k} acts on rows s .. s+b-1 with s = j + 1 + k b.  Two reflectors
// whose row ranges overlap must keep their relative order, and of two such
// reflectors the one of the lower sweep always comes first.  Grouping the
// reflectors of sweeps [J g, (J+1) g) at one step k into G(J, k), the product is
//   Q_b = prod_{J ascending} [ G(J, K) ... G(J, 1) G(J, 0) ],
//   G(J, k) = H_{Jg, k} H_{Jg+1, k} ... H_{Jg+g-1, k},
// because H_{j,k+1} precedes every overlapping H_{j',k} (j' > j), while H_{j,k}
// and H_{j',k+1} (j' >= j) never overlap.  So X <- Q_b X applies, for J
// descending, k ascending, the reflectors of G(J, k) with j descending -- the
// "bottom to top" group order of Sec. 2.1.2; within a group consecutive
// reflectors are one row apart, which keeps the rows of X in cache.
#include <algorithm>
#include <cstdio>

#include "device_util.cuh"
#include "evd_internal.h"

namespace evd {

namespace {

constexpr int BB_NT = 256;
constexpr int BB_NC = 64;  // columns of X per CTA

__host__ __device__ inline int64_t sweep_steps_b(int64_t n, int b, int64_t j) {
  if (j + 3 > n) return 0;
  return (n - 3 - j) / b + 1;
}
__host__ __device__ inline int64_t floor_sum_b(int64_t T, int b) {
  if (T < 0) return 0;
  int64_t q = T / b;
  return (int64_t)b * q * (q - 1) / 2 + q * (T - q * b + 1);
}
__host__ __device__ inline int64_t sweep_offset_b(int64_t n, int b, int64_t j) {
  int64_t jj = j < n - 2 ? j : (n - 2 > 0 ? n - 2 : 0);
  if (n < 3) return 0;
  return floor_sum_b(n - 3, b) - floor_sum_b(n - 3 - jj, b) + jj;
}

// One CTA per column strip; every CTA walks all reflectors in the valid order.
__global__ void __launch_bounds__(BB_NT) k_bc_back(const double* __restrict__ U, const double* __restrict__ Utau,
                                                   int64_t n, int b, int g, double* X, int64_t ldx) {
  __shared__ double v[128];
  const int64_t c0 = (int64_t)blockIdx.x * BB_NC;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nsweeps = (n >= 3) ? n - 2 : 0;
  const int64_t nJ = (nsweeps + g - 1) / g;
  for (int64_t J = nJ - 1; J >= 0; --J) {
    const int64_t j0 = J * g;
    const int64_t j1 = (j0 + g < nsweeps) ? j0 + g : nsweeps;  // sweeps [j0, j1)
    const int64_t kmax = sweep_steps_b(n, b, j0);              // the first sweep has the most steps
    for (int64_t k = 0; k < kmax; ++k) {
      for (int64_t j = j1 - 1; j >= j0; --j) {
        if (k >= sweep_steps_b(n, b, j)) continue;
        const int64_t idx = sweep_offset_b(n, b, j) + k;
        const double tau = Utau[idx];
        if (tau == 0.0) continue;
        const int64_t r0 = j + 1 + k * b;
        const int m = (int)((r0 + b - 1 < n - 1) ? b : n - r0);
        __syncthreads();
        if (threadIdx.x < b) v[threadIdx.x] = U[idx * b + threadIdx.x];
        __syncthreads();
        for (int cc = warp; cc < BB_NC; cc += BB_NT / 32) {
          const int64_t c = c0 + cc;
          if (c >= n) break;
          double* col = X + r0 + c * ldx;
          double s = 0.0;
          for (int t = lane; t < m; t += 32) s += v[t] * col[t];
          s = warp_sum(s) * tau;
          for (int t = lane; t < m; t += 32) col[t] -= s * v[t];
        }
      }
    }
  }
}

// Explicit V of SBR panel p: V(r, i) = 0 (r < i), 1 (r == i), A(r0 + r, c0 + i) (r > i).
__global__ void k_explicit_v(const double* A, int64_t lda, int64_t r0, int64_t c0, int64_t m, int kb, double* V,
                             int64_t ldv) {
  const int i = blockIdx.y;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    double x = (r < i) ? 0.0 : (r == i ? 1.0 : A[(r0 + r) + (c0 + i) * lda]);
    V[r + (int64_t)i * ldv] = x;
  }
}

}  // namespace

evd_status_t bc_back_run(const PlanCore& pc, const BcWork& bw, double* Q, int64_t ldq, const BackWork& w) {
  (void)w;
  const int64_t n = pc.n;
  if (n < 3 || pc.b < 2) return EVD_OK;
  const unsigned grid = (unsigned)ceil_div(n, BB_NC);
  StatScope sc("bc_back", pc.stream, 4.0 * pc.b * (double)n * (double)bc_num_reflectors(n, pc.b));
  k_bc_back<<<grid, BB_NT, 0, pc.stream>>>(bw.U, bw.Utau, n, pc.b, pc.b, Q, ldq); count_launch();
  EVD_CUDA_TRY(cudaGetLastError());
  return EVD_OK;
}

evd_status_t sbr_back_run(const PlanCore& pc, const double* A, const double* sbr_T, const double* sbr_tau,
                          double* Q, int64_t ldq, const BackWork& w) {
  (void)sbr_tau;
  const int64_t n = pc.n, lda = pc.lda;
  const int b = pc.b;
  cudaStream_t s = pc.stream;
  // number of factored panels
  int64_t np = 0;
  while (n - (np * b + b) >= 2) ++np;
  for (int64_t p = np - 1; p >= 0; --p) {
    const int64_t c0 = p * b, r0 = c0 + b, m = n - r0;
    const int bw = (int)((n - c0 < b) ? n - c0 : b);
    const int kb = (int)((bw < m) ? bw : m);
    k_explicit_v<<<dim3((unsigned)std::min<int64_t>(ceil_div(m, 256), 64), (unsigned)kb), 256, 0, s>>>(
        A, lda, r0, c0, m, kb, w.Vp, n); count_launch();
    EVD_CUDA_TRY(cudaGetLastError());
    // Wp = V^T X(r0:, :)   (kb x n)
    Gemm g1;
    g1.status = pc.status;
    g1.ta = 'T'; g1.m = kb; g1.n = n; g1.k = m; g1.A = w.Vp; g1.lda = n; g1.B = Q + r0; g1.ldb = ldq;
    g1.C = w.Wp; g1.ldc = b; g1.alpha = 1.0; g1.beta = 0.0;
    evd_status_t st = gemm(g1, pc.slices, w.gemm_ws, w.gemm_ws_bytes, s);
    if (st != EVD_OK) return st;
    // Tp = T Wp  (kb x n), T upper triangular kb x kb (ld b)
    Gemm g2;
    g2.status = pc.status;
    g2.m = kb; g2.n = n; g2.k = kb; g2.A = sbr_T + (size_t)p * b * b; g2.lda = b; g2.B = w.Wp; g2.ldb = b;
    g2.C = w.Tp; g2.ldc = b; g2.alpha = 1.0; g2.beta = 0.0;
    st = gemm(g2, 0, nullptr, 0, s);
    if (st != EVD_OK) return st;
    // X(r0:, :) -= V Tp
    Gemm g3;
    g3.status = pc.status;
    g3.m = m; g3.n = n; g3.k = kb; g3.A = w.Vp; g3.lda = n; g3.B = w.Tp; g3.ldb = b;
    g3.C = Q + r0; g3.ldc = ldq; g3.alpha = -1.0; g3.beta = 1.0;
    st = gemm(g3, pc.slices, w.gemm_ws, w.gemm_ws_bytes, s);
    if (st != EVD_OK) return st;
  }
  return EVD_OK;
}

}  // namespace evd
