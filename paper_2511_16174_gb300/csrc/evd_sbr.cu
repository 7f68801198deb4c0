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
#include <algorithm>
#include <cstdio>

#include "device_util.cuh"
#include "evd_internal.h"
#include "evd_ozaki.h"

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

// T (larft, forward columnwise) and W = V T after the panel QR, shared by both
// panel kernels.  Gram entries V(:, p)^T V(:, q), p < q, one warp each over all
// CTAs; CTA 0 forms T in shared memory; every CTA then copies T to shared memory
// and forms its rows of W.  Vs (optional) holds the CTA's rows of the in-place V
// (column-major, ld ldr); otherwise V is read from a.V.  Tsm: kb*kb doubles,
// Gsm: kb doubles (one Gram column at a time).
__device__ bool panel_finish_TW(const PanelArgs& a, unsigned G, int g, int64_t rb, int nr, const double* Vs, int ldr,
                                double* Tsm, double* Gsm, double* gram, double* sh_tmp) {
  const int kb = a.kb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (!grid_barrier(a.bar, G, a.st, 300)) return false;
  for (int e = g * (PQ_NT / 32) + warp; e < kb * kb; e += G * (PQ_NT / 32)) {
    const int p = e % kb, q = e / kb;
    double s0 = 0.0;
    if (p < q)
      for (int64_t r = q + lane; r < a.m; r += 32)
        s0 += __ldcg(a.V + r + (int64_t)p * a.ldv) * __ldcg(a.V + r + (int64_t)q * a.ldv);
    s0 = warp_sum(s0);
    if (lane == 0) gram[e] = s0;
  }
  if (!grid_barrier(a.bar, G, a.st, 301)) return false;
  if (g == 0) {
    for (int j = 0; j < kb; ++j) {
      const double tj = __ldcg(a.tau + j);
      for (int l = threadIdx.x; l < j; l += PQ_NT) Gsm[l] = __ldcg(gram + l + j * kb);  // Gram column j
      __syncthreads();
      for (int p = threadIdx.x; p < j; p += PQ_NT) {
        double s0 = 0.0;
        for (int l = p; l < j; ++l) s0 += Tsm[p + l * kb] * Gsm[l];
        sh_tmp[p] = -tj * s0;
      }
      __syncthreads();
      for (int p = threadIdx.x; p < kb; p += PQ_NT) Tsm[p + j * kb] = (p < j) ? sh_tmp[p] : (p == j ? tj : 0.0);
      __syncthreads();
    }
    for (int e = threadIdx.x; e < kb * kb; e += PQ_NT) a.T[(e % kb) + (e / kb) * a.b] = Tsm[e];
  }
  if (!grid_barrier(a.bar, G, a.st, 302)) return false;
  for (int e = threadIdx.x; e < kb * kb; e += PQ_NT) Tsm[e] = __ldcg(a.T + (e % kb) + (e / kb) * a.b);
  __syncthreads();
  for (int r = threadIdx.x; r < nr; r += PQ_NT) {
    const int64_t R = rb + r;
    for (int j = 0; j < kb; ++j) {
      double s0 = 0.0;
      for (int l = 0; l <= j; ++l) {
        double vl;
        if (R < l) vl = 0.0;
        else if (R == l) vl = 1.0;
        else vl = Vs ? Vs[r + (size_t)l * ldr] : a.V[R + (int64_t)l * a.ldv];
        s0 += vl * Tsm[l + j * kb];
      }
      a.W[R + (int64_t)j * a.ldv] = s0;
    }
  }
  return true;
}

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
  extern __shared__ double pdyn[];  // kb*kb (T) + kb (a Gram column)
  panel_finish_TW(a, G, g, rb, (int)(re - rb), nullptr, 0, pdyn, pdyn + a.kb * a.kb, gram, sh_y);
}

// Shared-memory form of the same panel QR (panel width <= 64): each CTA keeps its
// rows of the panel in shared memory for the whole factorization (column-major,
// leading dimension ldr), so the per-column dot products and updates never wait
// on L2.  The owner of row i publishes the diagonal entry alpha through the same
// partial-sum array as the norms (all other CTAs contribute exact zeros).
__global__ void __launch_bounds__(PQ_NT) k_panel_qr_smem(const PanelArgs a) {
  extern __shared__ double ps[];
  __shared__ double sh_y[128];
  __shared__ double sh_par[4];
  const unsigned G = gridDim.x;
  const int g = blockIdx.x;
  const int64_t chunk = (a.m + G - 1) / G;
  const int64_t rb = g * chunk, re = (rb + chunk < a.m) ? rb + chunk : a.m;
  const int nr = (int)(re > rb ? re - rb : 0);
  const int ldr = (int)chunk | 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int stride = 2 + a.bw;  // [norm, alpha, y_0 .. y_{bw-1}]
  double* part0 = a.partial;
  double* part1 = a.partial + (size_t)G * stride;
  double* gram = a.partial + 2 * (size_t)G * stride;
  // load own rows
  for (int j = 0; j < a.bw; ++j)
    for (int r = threadIdx.x; r < nr; r += PQ_NT) ps[r + j * ldr] = a.P[rb + r + (int64_t)j * a.lda];
  __syncthreads();
  // partial norm of column 0 below the diagonal, and alpha from the owner of row 0
  if (warp == 0) {
    double ss = 0.0;
    for (int r = lane; r < nr; r += 32) if (rb + r > 0) { const double x = ps[r]; ss += x * x; }
    ss = warp_sum(ss);
    if (lane == 0) {
      part0[(size_t)g * stride] = ss;
      part0[(size_t)g * stride + 1] = (rb == 0 && nr > 0) ? ps[0] : 0.0;
    }
  }
  for (int i = 0; i < a.kb; ++i) {
    double* cur = (i & 1) ? part1 : part0;
    double* nxt = (i & 1) ? part0 : part1;
    if (!grid_barrier(a.bar, G, a.st, 400 + i)) return;
    if (warp == 0) {
      double ss = 0.0, al = 0.0;
      for (unsigned q = lane; q < G; q += 32) {
        ss += __ldcg(cur + (size_t)q * stride);
        al += __ldcg(cur + (size_t)q * stride + 1);
      }
      ss = warp_sum(ss);
      al = warp_sum(al);
      if (lane == 0) {
        double tau = 0.0, beta = al, scale = 0.0;
        if (ss != 0.0) {
          const double nrm = sqrt(al * al + ss);
          beta = (al >= 0.0) ? -nrm : nrm;
          tau = (beta - al) / beta;
          scale = 1.0 / (al - beta);
        }
        sh_par[0] = tau; sh_par[1] = beta; sh_par[2] = scale;
      }
    }
    __syncthreads();
    const double tau = sh_par[0], scale = sh_par[2];
    const int lo = (rb > i) ? 0 : (int)(i - rb);  // first own row with global index >= i
    double* ci = ps + (size_t)i * ldr;
    // v in place below the diagonal (v_i = 1 implied at row i)
    for (int r = lo + threadIdx.x; r < nr; r += PQ_NT)
      if (rb + r > i) ci[r] *= scale;
    __syncthreads();
    // partial dots y_j = v^T P(:, j), j > i, over own rows >= i (one warp per column)
    for (int j = i + 1 + warp; j < a.bw; j += PQ_NT / 32) {
      const double* cj = ps + (size_t)j * ldr;
      double s0 = 0.0;
      for (int r = lo + lane; r < nr; r += 32) s0 += ((rb + r == i) ? 1.0 : ci[r]) * cj[r];
      s0 = warp_sum(s0);
      if (lane == 0) cur[(size_t)g * stride + 2 + j] = s0;
    }
    if (!grid_barrier(a.bar, G, a.st, 500 + i)) return;
    for (int j = i + 1 + warp; j < a.bw; j += PQ_NT / 32) {
      double s0 = 0.0;
      for (unsigned q = lane; q < G; q += 32) s0 += __ldcg(cur + (size_t)q * stride + 2 + j);
      s0 = warp_sum(s0);
      if (lane == 0) sh_y[j] = tau * s0;
    }
    __syncthreads();
    // update own rows of the remaining columns (row-parallel, columns in the loop)
    for (int r = lo + threadIdx.x; r < nr; r += PQ_NT) {
      const double vr = (rb + r == i) ? 1.0 : ci[r];
      for (int j = i + 1; j < a.bw; ++j) ps[r + (size_t)j * ldr] -= sh_y[j] * vr;
    }
    if (rb <= i && i < re && threadIdx.x == 0) {
      ci[i - rb] = sh_par[1];
      a.tau[i] = tau;
    }
    __syncthreads();
    // next column: partial norm below its diagonal and alpha from its owner
    if (i + 1 < a.kb && warp == 0) {
      const double* cn = ps + (size_t)(i + 1) * ldr;
      double ss = 0.0;
      for (int r = lane; r < nr; r += 32) if (rb + r > i + 1) { const double x = cn[r]; ss += x * x; }
      ss = warp_sum(ss);
      if (lane == 0) {
        nxt[(size_t)g * stride] = ss;
        nxt[(size_t)g * stride + 1] = (rb <= i + 1 && i + 1 < re) ? cn[i + 1 - rb] : 0.0;
      }
    }
  }
  // write back R / V, explicit V
  for (int j = 0; j < a.bw; ++j)
    for (int r = threadIdx.x; r < nr; r += PQ_NT) {
      const int64_t R = rb + r;
      const double x = ps[r + (size_t)j * ldr];
      a.P[R + (int64_t)j * a.lda] = x;
      if (j < a.kb) a.V[R + (int64_t)j * a.ldv] = (R < j) ? 0.0 : (R == j ? 1.0 : x);
    }
  double* Tsm = ps + (size_t)ldr * a.bw;
  panel_finish_TW(a, G, g, rb, nr, ps, ldr, Tsm, Tsm + a.kb * a.kb, gram, sh_y);
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

// Double-blocked SBR (DBBR, cited for Sec. 4.1): within a block of nb/b panels the
// trailing matrix is not updated; panel p instead
//   1. applies the block's pending update to its own columns,
//        A(c0:, c0:c0+b) -= [V Z]_< [Z V]_<^T,
//   2. is factored (panel QR, T, W),
//   3. forms Z = A2_stale W - V_< (Z_<^T W) - Z_< (V_<^T W), then Z -= 1/2 V (W^T Z),
// and the block ends with one rank-2 acc update of the trailing lower triangle,
//   A(c:, c:) -= [V Z] [Z V]^T   (K = 2 acc).
// The pending factors are kept interleaved per panel, VZ = [V_0 Z_0 V_1 Z_1 ...] and
// ZV = [Z_0 V_0 Z_1 V_1 ...], so that [V Z][Z V]^T = sum_q V_q Z_q^T + Z_q V_q^T is a
// single product.  With nb = b this is the plain Eq. 1 algorithm.
evd_status_t sbr_run(const PlanCore& pc, double* A, const SbrWork& w) {
  const int64_t n = pc.n, lda = pc.lda;
  const int b = pc.b;
  const int nbp = std::max(1, pc.nb / b);  // panels per block
  cudaStream_t s = pc.stream;
  {
    evd_status_t st = ensure_dynamic_smem((const void*)k_panel_qr, (size_t)(b * b + b) * 8);
    if (st == EVD_OK) st = ensure_dynamic_smem((const void*)k_panel_qr_smem, 200 * 1024);
    if (st != EVD_OK) return st;
  }
  int maxG = max_coresident_blocks((const void*)k_panel_qr, PQ_NT, (b * b + b) * 8);
  if (maxG < 1) return EVD_ERR_CUDA;
  const int maxG_smem = max_coresident_blocks((const void*)k_panel_qr_smem, PQ_NT, 200 * 1024);
  const int64_t ldz = n;  // leading dimension of VZ, ZV
  // scratch of the products; during a block with a presplit trailing matrix, what
  // follows the presplit
  char* gws = static_cast<char*>(w.gemm_ws);
  size_t gws_bytes = w.gemm_ws_bytes;
  auto gemm_tag = [&](Gemm g, const char* tag, bool tc) {
    g.status = pc.status;
    g.tag = tag;
    return gemm(g, tc ? pc.sbr_slices : 0, gws, gws_bytes, s);
  };
  // The Z products of one block all read principal submatrices of the block's
  // stale trailing matrix A(r0:, r0:): with more than one panel per block it is
  // split into slices once, at the block's start, when the scratch holds it next to
  // the largest product a panel runs.
  const size_t panel_scratch =
      std::max({gemm_scratch_bytes(n, b, 2 * (int64_t)pc.nb, pc.sbr_slices), gemm_scratch_bytes(2 * (int64_t)pc.nb, b, n, pc.sbr_slices),
                pc.sbr_slices > 0 ? ozaki_presplit_gemm_bytes(n, b, pc.sbr_slices) : (size_t)0});
  int64_t p = 0;
  bool done = false;
  while (!done) {
    int acc = 0;  // columns of V (and of Z) accumulated in this block
    SplitOperand pre;
    bool use_pre = false;
    gws = static_cast<char*>(w.gemm_ws);
    gws_bytes = w.gemm_ws_bytes;
    {
      const int64_t r0b = p * b + b, mb = n - r0b;
      if (nbp > 1 && b % 16 == 0 && pc.sbr_slices > 0 && mb >= 2 * b && mb <= ((int64_t)1 << 17)) {
        Gemm probe;
        probe.m = mb; probe.n = b; probe.k = mb;
        const size_t need = align_up(ozaki_presplit_bytes(mb, pc.sbr_slices), 256);
        if (ozaki_eligible(probe) && need + panel_scratch <= w.gemm_ws_bytes) {
          const evd_status_t st = ozaki_presplit_sym(A + r0b + r0b * lda, lda, mb, pc.sbr_slices, w.gemm_ws, need, "sbr_z",
                                                     &pre, s);
          if (st != EVD_OK) return st;
          use_pre = true;
          gws = static_cast<char*>(w.gemm_ws) + need;
          gws_bytes = w.gemm_ws_bytes - need;
        }
      }
    }
    const int64_t r0_block = p * b + b;
    for (int q = 0; q < nbp; ++q) {
      const int64_t c0 = p * b, r0 = c0 + b, m = n - r0;
      if (m < 2) { done = true; break; }
      const int bw = (int)((n - c0 < b) ? n - c0 : b);
      const int kb = (int)((bw < m) ? bw : m);
      evd_status_t st;
      // ---- 1. pending update of this panel's columns
      if (acc > 0) {
        Gemm g;
        g.tb = 'T'; g.m = n - c0; g.n = bw; g.k = 2 * acc;
        g.A = w.VZ + c0; g.lda = ldz; g.B = w.ZV + c0; g.ldb = ldz;
        g.C = A + c0 + c0 * lda; g.ldc = lda; g.alpha = -1.0; g.beta = 1.0;
        st = gemm_tag(g, "sbr_panel_update", true);
        if (st != EVD_OK) return st;
      }
      // ---- 2. panel QR, T, W
      {
        double* P = A + r0 + c0 * lda;
        PanelArgs pa;
        pa.P = P; pa.lda = lda; pa.m = m; pa.bw = bw; pa.kb = kb; pa.b = b;
        pa.tau = w.tau + c0;
        pa.V = w.V; pa.W = w.W; pa.ldv = n;
        pa.T = w.T + (size_t)p * b * b;
        pa.partial = w.partial; pa.bar = w.bar; pa.st = pc.status;
        EVD_CUDA_TRY(cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s));
        void* args[] = {&pa};
        StatScope sc("sbr_panel_qr", s, 4.0 * (double)m * bw * bw);
        const int64_t max_rows = (200 * 1024 - 8 * ((int64_t)kb * kb + kb)) / (8 * (int64_t)bw) - 1;
        // rows per CTA: at least 128 (a column step is a norm and a rank-1 update of
        // the CTA's rows, far below a grid barrier's cost), so small panels take few
        // CTAs and leave the rest of the GPU to concurrent solves
        int Gs = (int)std::max<int64_t>(ceil_div(m, max_rows), std::min<int64_t>(ceil_div(m, 128), pc.sms));
        if (bw <= 64 && Gs <= pc.sms && Gs <= maxG_smem) {
          const int64_t chunk = ceil_div(m, Gs);
          const size_t smem = ((size_t)(chunk | 1) * bw + (size_t)kb * kb + kb) * sizeof(double);
          EVD_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_panel_qr_smem, dim3(Gs), dim3(PQ_NT), args, smem, s)); count_launch();
        } else {
          int G = (int)ceil_div(m, 64);
          if (G > pc.panel_ctas) G = pc.panel_ctas;  // barrier cost grows with the CTA count
          if (G > maxG) G = maxG;
          if (G < 1) G = 1;
          EVD_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_panel_qr, dim3(G), dim3(PQ_NT), args,
                                                   ((size_t)kb * kb + kb) * sizeof(double), s)); count_launch();
        }
      }
      double* A2 = A + r0 + r0 * lda;
      // ---- 3. Y = A2_stale W - [V Z]_< ([Z V]_<^T W)
      {
        Gemm g;
        g.m = m; g.n = kb; g.k = m; g.A = A2; g.lda = lda; g.a_sym_lower = true;
        g.B = w.W; g.ldb = n; g.C = w.Y; g.ldc = n; g.alpha = 1.0; g.beta = 0.0;
        if (use_pre && ozaki_eligible(g) && r0 - r0_block + m == pre.rows) {
          g.a_sym_lower = false;  // the presplit holds the mirrored matrix
          g.status = pc.status;
          g.tag = "sbr_z";
          st = ozaki_gemm_presplit(g, pre, r0 - r0_block, gws, gws_bytes, s);
        } else {
          st = gemm_tag(g, "sbr_z", true);
        }
        if (st != EVD_OK) return st;
      }
      if (acc > 0) {
        Gemm g;
        g.ta = 'T'; g.m = 2 * acc; g.n = kb; g.k = m; g.A = w.ZV + r0; g.lda = ldz; g.B = w.W; g.ldb = n;
        g.C = w.X; g.ldc = 2 * pc.nb; g.alpha = 1.0; g.beta = 0.0;
        st = gemm_tag(g, "sbr_z_corr", 2 * acc > 128);
        if (st != EVD_OK) return st;
        Gemm g2;
        g2.m = m; g2.n = kb; g2.k = 2 * acc; g2.A = w.VZ + r0; g2.lda = ldz; g2.B = w.X; g2.ldb = 2 * pc.nb;
        g2.C = w.Y; g2.ldc = n; g2.alpha = -1.0; g2.beta = 1.0;
        st = gemm_tag(g2, "sbr_z_corr", true);
        if (st != EVD_OK) return st;
      }
      // ---- M = W^T Y ; Z = Y - 1/2 V M
      {
        Gemm g;
        g.ta = 'T'; g.m = kb; g.n = kb; g.k = m; g.A = w.W; g.lda = n; g.B = w.Y; g.ldb = n;
        g.C = w.M; g.ldc = b; g.alpha = 1.0; g.beta = 0.0;
        st = gemm_tag(g, "sbr_small", false);
        if (st != EVD_OK) return st;
        // Z (appended to VZ / ZV below) = Y - 1/2 V M
        EVD_CUDA_TRY(cudaMemcpy2DAsync(w.Z, n * sizeof(double), w.Y, n * sizeof(double), m * sizeof(double), kb,
                                       cudaMemcpyDeviceToDevice, s));
        Gemm g3;
        g3.m = m; g3.n = kb; g3.k = kb; g3.A = w.V; g3.lda = n; g3.B = w.M; g3.ldb = b; g3.C = w.Z; g3.ldc = n;
        g3.alpha = -0.5; g3.beta = 1.0;
        st = gemm_tag(g3, "sbr_small", false);
        if (st != EVD_OK) return st;
      }
      // ---- append V_p, Z_p (rows r0.. ; rows above r0 zero) to VZ / ZV
      {
        double* vz_v = w.VZ + (size_t)(2 * acc) * ldz;
        double* vz_z = w.VZ + (size_t)(2 * acc + kb) * ldz;
        double* zv_z = w.ZV + (size_t)(2 * acc) * ldz;
        double* zv_v = w.ZV + (size_t)(2 * acc + kb) * ldz;
        EVD_CUDA_TRY(cudaMemset2DAsync(vz_v, ldz * sizeof(double), 0, r0 * sizeof(double), 2 * kb, s));
        EVD_CUDA_TRY(cudaMemset2DAsync(zv_z, ldz * sizeof(double), 0, r0 * sizeof(double), 2 * kb, s));
        if ((st = copy_matrix(w.V, n, vz_v + r0, ldz, m, kb, s)) != EVD_OK) return st;
        if ((st = copy_matrix(w.Z, n, vz_z + r0, ldz, m, kb, s)) != EVD_OK) return st;
        if ((st = copy_matrix(w.Z, n, zv_z + r0, ldz, m, kb, s)) != EVD_OK) return st;
        if ((st = copy_matrix(w.V, n, zv_v + r0, ldz, m, kb, s)) != EVD_OK) return st;
        acc += kb;
      }
      // ---- band of this column block is final
      k_pack_band<<<bw, 128, 0, s>>>(A, lda, n, b, w.band, c0, c0 + bw, c0, 1); count_launch();
      EVD_CUDA_TRY(cudaGetLastError());
      ++p;
    }
    // ---- block end: trailing lower triangle from column c = p b (the presplit is
    // stale from here on; the whole scratch is free again)
    gws = static_cast<char*>(w.gemm_ws);
    gws_bytes = w.gemm_ws_bytes;
    const int64_t c = p * b;
    if (acc > 0 && c < n) {
      Gemm g;
      g.tb = 'T'; g.m = n - c; g.n = n - c; g.k = 2 * acc; g.A = w.VZ + c; g.lda = ldz; g.B = w.ZV + c; g.ldb = ldz;
      g.C = A + c + c * lda; g.ldc = lda; g.alpha = -1.0; g.beta = 1.0; g.lower = true;
      evd_status_t st = gemm_tag(g, "sbr_syr2k", true);
      if (st != EVD_OK) return st;
    }
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
