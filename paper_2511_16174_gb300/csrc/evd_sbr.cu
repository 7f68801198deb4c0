// Successive band reduction (Sec. 2.1.1, Eq. 1) on one GB300.
//
// For each panel p (columns c0 = p b .. c0 + b - 1) the panel below the band,
// P = A(r0:n, c0:c0+b) with r0 = c0 + b, is factored by Householder QR,
// QR(P) = (I - W Y^T) R with W = Y T, by a cooperative kernel in which every CTA owns
// a contiguous slice of the panel rows (two grid barriers per column).  The
// trailing matrix A2 = A(r0:n, r0:n) (lower triangle stored) then gets the ZY
// update of Eq. 1:
//     Z  = A2 W - 1/2 Y (W^T A2 W)
//     A2 = A2 - Y Z^T - Z Y^T      (lower triangle only)
// through the dense-product engine.  After panel p, columns c0.. of the band are
// final and are packed into the band storage the bulge chasing reads; with
// EVD_VECTORS the Householder vectors stay in A below the band and T in the
// workspace for SBR-Back.
#include <cstdio>

#include "device_util.cuh"
#include "evd_internal.h"

namespace evd {

namespace {

constexpr int PQ_NT = 256;

struct PanelArgs {
  double* P;      // panel top-left, A(r0, c0)
  int64_t lda;
  int64_t m;      // rows
  int bw;         // columns
  int kb;         // reflectors = min(bw, m)
  int b;          // ld of T
  double* tau;    // kb
  double* V;      // explicit V, m x kb, ld ldv
  double* W;      // W = V T, m x kb, ld ldv
  int64_t ldv;
  double* T;      // kb x kb, ld b
  double* partial;  // [2][G][1 + bw] then gram scratch [kb*kb]
  unsigned* bar;
  int* st;
};

// Householder QR of the m x bw panel, then T and W = V T.  Cooperative launch.
// Values another CTA wrote (partial sums, the diagonal entry, V, the Gram matrix,
// T, tau) are read through L2 (ld.cg) after the grid barrier.
__global__ void __launch_bounds__(PQ_NT) k_panel_qr(const PanelArgs a) {
  __shared__ double red[PQ_NT];
  __shared__ double sh_y[128];
  __shared__ double sh_par[4];
  const unsigned G = gridDim.x;
  const int g = blockIdx.x;
  const int64_t chunk = (a.m + G - 1) / G;
  const int64_t rb = g * chunk, re = (rb + chunk < a.m) ? rb + chunk : a.m;
  const int stride = 1 + a.bw;
  double* part0 = a.partial;
  double* part1 = a.partial + (size_t)G * stride;
  double* gram = a.partial + 2 * (size_t)G * stride;

  // norm^2 of column 0 below the diagonal
  {
    double ss = 0.0;
    for (int64_t r = rb + threadIdx.x; r < re; r += PQ_NT)
      if (r > 0) { double x = a.P[r]; ss += x * x; }
    ss = block_sum<PQ_NT>(ss, red);
    if (threadIdx.x == 0) part0[(size_t)g * stride] = ss;
  }
  for (int i = 0; i < a.kb; ++i) {
    double* cur = (i & 1) ? part1 : part0;
    double* nxt = (i & 1) ? part0 : part1;
    if (!grid_barrier(a.bar, G, a.st, 100 + i)) return;
    // ---- reflector for column i (every CTA computes the same scalars)
    if (threadIdx.x < 32) {
      // the per-CTA partial norms, summed by one warp (lanes load in parallel)
      double ss = 0.0;
      for (unsigned q = threadIdx.x; q < G; q += 32) ss += __ldcg(cur + (size_t)q * stride);
      ss = warp_sum(ss);
      if (threadIdx.x == 0) {
      double alpha = __ldcg(a.P + i + (int64_t)i * a.lda);
      double tau = 0.0, beta = alpha, scale = 0.0;
      if (ss != 0.0) {
        double nrm = sqrt(alpha * alpha + ss);
        beta = (alpha >= 0.0) ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      sh_par[0] = tau; sh_par[1] = beta; sh_par[2] = scale;
      }
    }
    __syncthreads();
    const double tau = sh_par[0], scale = sh_par[2];
    double* col = a.P + (int64_t)i * a.lda;
    // v below the diagonal (in place) and explicit V
    for (int64_t r = rb + threadIdx.x; r < re; r += PQ_NT) {
      double v;
      if (r > i) { v = col[r] * scale; col[r] = v; }
      else v = (r == i) ? 1.0 : 0.0;
      a.V[r + (int64_t)i * a.ldv] = v;
    }
    __syncthreads();
    // partial dots y_j = v^T P(:, j) for j > i over own rows (r >= i), one warp per column
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int j = i + 1 + warp; j < a.bw; j += PQ_NT / 32) {
        const double* pj = a.P + (int64_t)j * a.lda;
        double s = 0.0;
        for (int64_t r = (rb > i ? rb : i) + lane; r < re; r += 32) s += a.V[r + (int64_t)i * a.ldv] * pj[r];
        s = warp_sum(s);
        if (lane == 0) cur[(size_t)g * stride + 1 + j] = s;
      }
    }
    if (!grid_barrier(a.bar, G, a.st, 200 + i)) return;
    {
      // y_j = sum of the per-CTA partials, one warp per column
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int j = i + 1 + warp; j < a.bw; j += PQ_NT / 32) {
        double s = 0.0;
        for (unsigned q = lane; q < G; q += 32) s += __ldcg(cur + (size_t)q * stride + 1 + j);
        s = warp_sum(s);
        if (lane == 0) sh_y[j] = s;
      }
    }
    __syncthreads();
    // update own rows of the remaining columns
    for (int j = i + 1; j < a.bw; ++j) {
      double* pj = a.P + (int64_t)j * a.lda;
      const double ty = tau * sh_y[j];
      for (int64_t r = (rb > i ? rb : i) + threadIdx.x; r < re; r += PQ_NT)
        pj[r] -= ty * a.V[r + (int64_t)i * a.ldv];
    }
    if (rb <= i && i < re && threadIdx.x == 0) {
      col[i] = sh_par[1];
      a.tau[i] = tau;
    }
    // norm^2 of the next column below its diagonal (rows updated above by other threads)
    __syncthreads();
    if (i + 1 < a.kb && threadIdx.x < 32) {
      const double* pn = a.P + (int64_t)(i + 1) * a.lda;
      double ss = 0.0;
      for (int64_t r = rb + threadIdx.x; r < re; r += 32)
        if (r > i + 1) { double x = pn[r]; ss += x * x; }
      ss = warp_sum(ss);
      if (threadIdx.x == 0) nxt[(size_t)g * stride] = ss;
    }
  }
  // ---- Gram matrix V^T V: each CTA reduces the entries e with e % G == g
  if (!grid_barrier(a.bar, G, a.st, 300)) return;
  const int kb = a.kb;
  for (int e = g; e < kb * kb; e += G) {
    int p = e % kb, q = e / kb;
    double s = 0.0;
    if (p < q) {
      for (int64_t r = q + threadIdx.x; r < a.m; r += PQ_NT)
        s += __ldcg(a.V + r + (int64_t)p * a.ldv) * __ldcg(a.V + r + (int64_t)q * a.ldv);
    }
    s = block_sum<PQ_NT>(s, red);
    if (threadIdx.x == 0) gram[e] = s;
  }
  if (!grid_barrier(a.bar, G, a.st, 301)) return;
  // ---- T (forward, columnwise): T(0:j, j) = -tau_j T(0:j, 0:j) gram(0:j, j), CTA 0
  if (g == 0) {
    double* T = a.T;
    for (int j = 0; j < kb; ++j) {
      double tj = __ldcg(a.tau + j);
      if (threadIdx.x == 0) T[j + j * a.b] = tj;
      for (int p = threadIdx.x; p < j; p += PQ_NT) {
        double s = 0.0;
        for (int l = p; l < j; ++l) s += T[p + l * a.b] * __ldcg(gram + l + j * kb);
        sh_y[p] = -tj * s;
      }
      __syncthreads();
      for (int p = threadIdx.x; p < j; p += PQ_NT) T[p + j * a.b] = sh_y[p];
      for (int p = j + 1 + threadIdx.x; p < kb; p += PQ_NT) T[p + j * a.b] = 0.0;
      __syncthreads();
    }
  }
  if (!grid_barrier(a.bar, G, a.st, 302)) return;
  // ---- W = V T over own rows
  for (int64_t idx = threadIdx.x; idx < (re - rb) * kb; idx += PQ_NT) {
    int64_t r = rb + idx % (re - rb);
    int j = (int)(idx / (re - rb));
    double s = 0.0;
    for (int l = 0; l <= j; ++l) s += a.V[r + (int64_t)l * a.ldv] * __ldcg(a.T + l + j * a.b);
    a.W[r + (int64_t)j * a.ldv] = s;
  }
}

// Pack columns [c_begin, c_end) of the band into band storage (ldb = 2b + 1):
// band[(r - c) + c ldb] = B(r, c) for 0 <= r - c <= b, zero for b < r - c <= 2b.
// Columns of a factored panel (c0 = panel start) keep R's upper triangle at rows
// r0 = c0 + b .. and drop the Householder vectors below it.
__global__ void k_pack_band(const double* __restrict__ A, int64_t lda, int64_t n, int b, double* band,
                            int64_t c_begin, int64_t c_end, int64_t c0, int factored) {
  int64_t c = c_begin + blockIdx.x;
  if (c >= c_end) return;
  const int ldb = 2 * b + 1;
  for (int o = threadIdx.x; o < ldb; o += blockDim.x) {
    int64_t r = c + o;
    double v = 0.0;
    if (o <= b && r < n) {
      v = A[r + c * lda];
      if (factored) {
        int64_t r0 = c0 + b;
        if (r >= r0 && (r - r0) > (c - c0)) v = 0.0;
      }
    }
    band[o + c * ldb] = v;
  }
}

}  // namespace

evd_status_t sbr_run(const PlanCore& pc, double* A, const SbrWork& w) {
  const int64_t n = pc.n, lda = pc.lda;
  const int b = pc.b;
  cudaStream_t s = pc.stream;
  int maxG = max_coresident_blocks((const void*)k_panel_qr, PQ_NT, 0);
  if (maxG < 1) return EVD_ERR_CUDA;
  int64_t p = 0;
  for (;; ++p) {
    const int64_t c0 = p * b, r0 = c0 + b, m = n - r0;
    if (m < 2) break;
    const int bw = (int)((n - c0 < b) ? n - c0 : b);
    const int kb = (int)((bw < m) ? bw : m);
    double* P = A + r0 + c0 * lda;
    // ---- panel QR, T, W
    PanelArgs pa;
    pa.P = P; pa.lda = lda; pa.m = m; pa.bw = bw; pa.kb = kb; pa.b = b;
    pa.tau = w.tau + c0;
    pa.V = w.V; pa.W = w.W; pa.ldv = n;
    pa.T = w.T + (size_t)p * b * b;
    pa.partial = w.partial; pa.bar = w.bar; pa.st = pc.status;
    int G = (int)ceil_div(m, 64);
    if (G > pc.panel_ctas) G = pc.panel_ctas;  // barrier cost grows with the CTA count
    if (G > maxG) G = maxG;
    if (G < 1) G = 1;
    EVD_CUDA_TRY(cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s));
    void* args[] = {&pa};
    StatScope sc("sbr_panel_qr", s, 4.0 * (double)m * bw * bw);
    EVD_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_panel_qr, dim3(G), dim3(PQ_NT), args, 0, s)); count_launch();
    // ---- Eq. 1: Y = A2 W ; M = W^T Y ; Z = Y - 1/2 V M ; A2 -= V Z^T + Z V^T
    double* A2 = A + r0 + r0 * lda;
    Gemm g1;
    g1.status = pc.status;
    g1.m = m; g1.n = kb; g1.k = m; g1.A = A2; g1.lda = lda; g1.a_sym_lower = true;
    g1.B = w.W; g1.ldb = n; g1.C = w.Y; g1.ldc = n; g1.alpha = 1.0; g1.beta = 0.0;
    evd_status_t st = gemm(g1, pc.slices, w.gemm_ws, w.gemm_ws_bytes, s);
    if (st != EVD_OK) return st;
    Gemm g2;
    g2.status = pc.status;
    g2.ta = 'T'; g2.m = kb; g2.n = kb; g2.k = m; g2.A = w.W; g2.lda = n; g2.B = w.Y; g2.ldb = n;
    g2.C = w.M; g2.ldc = b; g2.alpha = 1.0; g2.beta = 0.0;
    st = gemm(g2, 0, w.gemm_ws, w.gemm_ws_bytes, s);
    if (st != EVD_OK) return st;
    EVD_CUDA_TRY(cudaMemcpy2DAsync(w.Z, n * sizeof(double), w.Y, n * sizeof(double), m * sizeof(double), kb,
                                   cudaMemcpyDeviceToDevice, s));
    Gemm g3;
    g3.status = pc.status;
    g3.m = m; g3.n = kb; g3.k = kb; g3.A = w.V; g3.lda = n; g3.B = w.M; g3.ldb = b; g3.C = w.Z; g3.ldc = n;
    g3.alpha = -0.5; g3.beta = 1.0;
    st = gemm(g3, 0, nullptr, 0, s);
    if (st != EVD_OK) return st;
    Gemm g4;
    g4.status = pc.status;
    g4.tb = 'T'; g4.m = m; g4.n = m; g4.k = kb; g4.A = w.V; g4.lda = n; g4.B = w.Z; g4.ldb = n;
    g4.C = A2; g4.ldc = lda; g4.alpha = -1.0; g4.beta = 1.0; g4.lower = true;
    st = gemm(g4, pc.slices, w.gemm_ws, w.gemm_ws_bytes, s);
    if (st != EVD_OK) return st;
    Gemm g5 = g4;
    g5.A = w.Z; g5.B = w.V;
    st = gemm(g5, pc.slices, w.gemm_ws, w.gemm_ws_bytes, s);
    if (st != EVD_OK) return st;
    // ---- band of this column block is final
    k_pack_band<<<bw, 128, 0, s>>>(A, lda, n, b, w.band, c0, c0 + bw, c0, 1); count_launch();
    EVD_CUDA_TRY(cudaGetLastError());
  }
  // remaining columns need no reduction
  const int64_t cstart = p * b;
  if (cstart < n) {
    k_pack_band<<<(unsigned)(n - cstart), 128, 0, s>>>(A, lda, n, b, w.band, cstart, n, cstart, 0); count_launch();
    EVD_CUDA_TRY(cudaGetLastError());
  }
  return EVD_OK;
}

}  // namespace evd
