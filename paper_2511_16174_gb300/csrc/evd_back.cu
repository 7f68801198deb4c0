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
//
// Wavefronts.  With g = b, G(J, k) touches rows [(J+k) b + 1, (J+k+2) b - 1], so two
// groups overlap exactly when their diagonal indices D = J + k differ by at most 1.
// Give G(J, k) the wave number t = k + (nJ - 1 - J).  Every overlapping pair keeps its
// order: the same J with k ascending raises t, and J1 > J2 with |D1 - D2| <= 1 gives
// k1 - k2 <= 1 - (J1 - J2) < J1 - J2, i.e. t1 < t2.  Two groups of one wave have
// D1 - D2 = 2 (J1 - J2), so they are disjoint (2b rows apart) and commute.  Each wave
// is therefore one batched pair of products: W_p^T = X_p^T V_p and X_p -= Y_p W_p,
// about 2n/b waves in all instead of n^2/(2 b g) separate groups.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstdio>
#include <vector>

#include "device_util.cuh"
#include "evd_internal.h"
#include "evd_ozaki.h"

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

// Compact WY factors of the BC reflector groups of one sweep block J: group k
// holds the reflectors (j, k), j in [J g, J g + g), whose rows lie in
// [R0, R0 + g + b - 1) with R0 = J g + 1 + k b; reflector j sits in column
// i = j - J g at rows i .. i + b - 1 of the group.  For each group the kernel forms
// V (h x g, explicit, zero outside the parallelogram), T (g x g upper triangular,
// H_{j0} ... H_{j0+g-1} = I - V T V^T) and Y = V T.  One CTA per group.
// Problem p of wave t is the group with J' = jp0 + p, J = nJ - 1 - J', k = t - J'.
__global__ void __launch_bounds__(256) k_bcback_prep(const double* __restrict__ U, const double* __restrict__ Utau,
                                                     int64_t n, int b, int g, int64_t nJ, int64_t t, int64_t jp0,
                                                     double* Vg, double* Yg, int h) {
  extern __shared__ double sp[];
  double* V = sp;                 // V[r + i h], h x g
  double* T = V + (size_t)h * g;  // T[p + i g]
  double* tau = T + (size_t)g * g;
  const int64_t pidx = blockIdx.x;
  const int64_t J = nJ - 1 - (jp0 + pidx), k = t - (jp0 + pidx);
  const int64_t nsweeps = n - 2;
  for (int idx = threadIdx.x; idx < h * g; idx += blockDim.x) V[idx] = 0.0;
  __syncthreads();
  for (int i = threadIdx.y; i < g; i += blockDim.y) {  // (blockDim = 32 x 8)
    const int64_t j = J * g + i;
    double t = 0.0;
    if (j < nsweeps && k < sweep_steps_b(n, b, j)) {
      const int64_t idx = sweep_offset_b(n, b, j) + k;
      t = Utau[idx];
      const int64_t r0 = j + 1 + k * b;
      const int m = (int)((r0 + b - 1 < n - 1) ? b : n - r0);
      for (int q = threadIdx.x; q < m; q += 32) V[(i + q) + (size_t)i * h] = U[idx * b + q];
    }
    if (threadIdx.x == 0) tau[i] = t;
  }
  __syncthreads();
  // T, column by column: T(0:i, i) = -tau_i T(0:i, 0:i) (V(:, 0:i)^T v_i)
  double* gv = T + (size_t)g * g + g;  // g scratch
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int i = 0; i < g; ++i) {
    const double ti = tau[i];
    for (int l = tid; l < i; l += 256) {
      double s = 0.0;
      const int lo = i, hi = (l + b - 1 < h - 1) ? l + b - 1 : h - 1;
      for (int r = lo; r <= hi; ++r) s += V[r + (size_t)l * h] * V[r + (size_t)i * h];
      gv[l] = s;
    }
    __syncthreads();
    for (int p = tid; p < g; p += 256) {
      double s = 0.0;
      if (p < i)
        for (int l = p; l < i; ++l) s += T[p + (size_t)l * g] * gv[l];
      T[p + (size_t)i * g] = (p < i) ? -ti * s : (p == i ? ti : 0.0);
    }
    __syncthreads();
  }
  // write V and Y = V T (h x g each, problem p at offset p h g)
  double* Vo = Vg + (size_t)pidx * h * g;
  double* Yo = Yg + (size_t)pidx * h * g;
  for (int idx = tid; idx < h * g; idx += 256) {
    const int r = idx % h, i = idx / h;
    double s = 0.0;
    for (int l = 0; l <= i; ++l) s += V[r + (size_t)l * h] * T[l + (size_t)i * g];
    Yo[idx] = s;
    Vo[idx] = V[idx];
  }
}

// Explicit V of SBR panel p inside a block of panels: rows [0, roff) of the block
// are zero, and below them V(r, i) = 0 (r < i), 1 (r == i), A(r0 + r, c0 + i)
// (r > i) with r counted from roff.  m = rows of the block.
__global__ void k_explicit_v(const double* A, int64_t lda, int64_t r0, int64_t c0, int64_t roff, int64_t m, int kb,
                             double* V, int64_t ldv) {
  const int i = blockIdx.y;
  for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < m; rr += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = rr - roff;
    double x = (r < i) ? 0.0 : (r == i ? 1.0 : A[(r0 + r) + (c0 + i) * lda]);
    V[rr + (int64_t)i * ldv] = x;
  }
}

}  // namespace

int64_t bc_wave_max_groups(int64_t n, int b) { return (b > 0) ? n / (2 * (int64_t)b) + 2 : 1; }

int64_t bc_num_groups(int64_t n, int b) {
  if (n < 3 || b < 2) return 0;
  const int64_t nJ = ceil_div(n - 2, b);
  int64_t total = 0;
  for (int64_t J = 0; J < nJ; ++J) total += sweep_steps_b(n, b, J * b);
  return total;
}

// The wave launches of the fused BC-Back in order (wave t, then the maximal runs of
// valid groups of that wave), each group's (J, k), and the identity start's column
// ranges.  Identity start: X = I at first, so row r is nonzero in column r only; a
// group mixes its rows, so afterwards all of them are nonzero at most over the union
// of their column ranges.  With g = b the group G(J, k) covers rows (J+k) b + 1 ..
// (J+k+2) b - 1, inside the b-row blocks q = J + k and q + 1 (block q: rows q b + 1
// .. q b + b), and the groups of one launch cover disjoint blocks, so tracking one
// column interval per block, in launch order, gives a superset of every group's
// support.
evd_status_t bb_schedule_build(int64_t n, int b, BbSchedule* out) {
  BbSchedule sc;
  const int g = b, h = g + b - 1;
  const int64_t nJ = ceil_div(n - 2, g);
  auto kc = [&](int64_t J) { return sweep_steps_b(n, b, J * g); };
  const int64_t tmax = kc(0) + nJ - 2;
  const int64_t nblk = n / b + 3;
  std::vector<int64_t> cmin(nblk), cmax(nblk);
  for (int64_t q = 0; q < nblk; ++q) {
    cmin[q] = std::min<int64_t>(q * b + 1, n - 1);
    cmax[q] = std::min<int64_t>(q * b + b, n - 1);
  }
  std::vector<int2> gjk, ranges;
  for (int64_t t = 0; t <= tmax; ++t) {
    int64_t jp = std::min<int64_t>(t, nJ - 1);
    while (jp >= 0) {
      if (t - jp >= kc(nJ - 1 - jp)) { --jp; continue; }
      const int64_t jhi = jp;
      while (jp >= 0 && t - jp < kc(nJ - 1 - jp)) --jp;
      const int64_t jlo = jp + 1;
      BbLaunch L;
      L.count = (int)(jhi - jlo + 1);
      // group 0 (J' = jlo) is the lowest group of the run and the only one that may reach row n
      L.R0 = (nJ - 1 - jlo) * g + 1 + (t - jlo) * b;
      L.hh0 = (int)std::min<int64_t>(h, n - L.R0);
      L.g0 = (int64_t)gjk.size();
      L.tile0 = INT64_MAX;
      L.tile1 = -1;
      L.work_tiles = 0;
      for (int64_t jq = jlo; jq <= jhi; ++jq) {
        const int64_t J = nJ - 1 - jq, k = t - jq, q = J + k;
        gjk.push_back(make_int2((int)J, (int)k));
        const int64_t lo = std::min(cmin[q], cmin[q + 1]), hi = std::max(cmax[q], cmax[q + 1]);
        cmin[q] = cmin[q + 1] = lo;
        cmax[q] = cmax[q + 1] = hi;
        const int2 r = make_int2((int)(lo / 128), (int)(hi / 128));
        ranges.push_back(r);
        L.tile0 = std::min<int64_t>(L.tile0, r.x);
        L.tile1 = std::max<int64_t>(L.tile1, r.y);
        L.work_tiles += r.y - r.x + 1;
      }
      sc.max_count = std::max(sc.max_count, L.count);
      sc.launches.push_back(L);
    }
  }
  sc.groups = (int64_t)gjk.size();
  const size_t bytes = sizeof(int2) * (size_t)std::max<int64_t>(sc.groups, 1);
  if (cudaMalloc(&sc.d_gjk, bytes) != cudaSuccess || cudaMalloc(&sc.d_ranges, bytes) != cudaSuccess) {
    bb_schedule_free(&sc);
    (void)cudaGetLastError();
    return EVD_ERR_OOM;
  }
  if (sc.groups > 0 &&
      (cudaMemcpy(sc.d_gjk, gjk.data(), sizeof(int2) * gjk.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(sc.d_ranges, ranges.data(), sizeof(int2) * ranges.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
    bb_schedule_free(&sc);
    return EVD_ERR_CUDA;
  }
  *out = std::move(sc);
  return EVD_OK;
}

void bb_schedule_free(BbSchedule* s) {
  if (!s) return;
  if (s->d_gjk) cudaFree(s->d_gjk);
  if (s->d_ranges) cudaFree(s->d_ranges);
  s->d_gjk = s->d_ranges = nullptr;
  s->launches.clear();
}

namespace {

// The fused waves in chunks: the group factors of as many consecutive launches as
// the scratch holds are prepared in one go, then those launches run.
evd_status_t fused_waves(const PlanCore& pc, const BcWork& bw, double* Q, int64_t ldq, const BackWork& w,
                         bool identity) {
  const BbSchedule& sc = *pc.bb;
  int64_t cmax = std::min<int64_t>(sc.groups, 65535);
  while (cmax > sc.max_count && bcback_prep_bytes((int)cmax, pc.ref_slices) > w.gemm_ws_bytes) cmax /= 2;
  cmax = std::max<int64_t>(cmax, sc.max_count);
  if (bcback_prep_bytes((int)cmax, pc.ref_slices) > w.gemm_ws_bytes)
    return ws_fail("bc_back fused prep", w.gemm_ws_bytes, bcback_prep_bytes((int)cmax, pc.ref_slices));
  size_t i = 0;
  while (i < sc.launches.size()) {
    const size_t first = i;
    int64_t cnt = 0;
    while (i < sc.launches.size() && cnt + sc.launches[i].count <= cmax) cnt += sc.launches[i++].count;
    const int64_t g_begin = sc.launches[first].g0;
    evd_status_t st = bcback_prep_chunk(pc, bw, sc.d_gjk + g_begin, (int)cnt, w.gemm_ws);
    if (st != EVD_OK) return st;
    for (size_t l = first; l < i; ++l) {
      const BbLaunch& L = sc.launches[l];
      WaveTiles wt;
      if (identity) {
        wt.ranges = sc.d_ranges + L.g0;
        wt.tile0 = L.tile0;
        wt.tile1 = L.tile1;
        wt.work_tiles = L.work_tiles;
      }
      st = bcback_fused_wave(pc, Q, ldq, w.gemm_ws, (int)cnt, (int)(L.g0 - g_begin), L.count, L.R0, L.hh0, wt);
      if (st != EVD_OK) return st;
    }
  }
  return EVD_OK;
}

}  // namespace

evd_status_t bc_back_run(const PlanCore& pc, const BcWork& bw, double* Q, int64_t ldq, const BackWork& w,
                         bool identity) {
  const int64_t n = pc.n;
  if (identity) {
    // BC-Back of the identity (reordered stages): X = I first
    const evd_status_t st = set_identity(Q, ldq, n, pc.stream);
    if (st != EVD_OK) return st;
  }
  if (n < 3 || pc.b < 2) return EVD_OK;
  const int b = pc.b, g = pc.b;
  const int h = g + b - 1;
  const size_t smem = ((size_t)h * g + (size_t)g * g + 2 * g) * sizeof(double);
  // small problems, and band widths whose group factors do not fit in shared
  // memory (b > 64): reflector-by-reflector kernel on FP64 cores
  if (pc.slices <= 0 || n < 256 || (!w.Vg && !identity) || smem > kMaxDynamicSmem) {
    const unsigned grid = (unsigned)ceil_div(n, BB_NC);
    StatScope sc("bc_back", pc.stream, 4.0 * pc.b * (double)n * (double)bc_num_reflectors(n, pc.b));
    k_bc_back<<<grid, BB_NT, 0, pc.stream>>>(bw.U, bw.Utau, n, pc.b, pc.b, Q, ldq); count_launch();
    EVD_CUDA_TRY(cudaGetLastError());
    return EVD_OK;
  }
  cudaStream_t s = pc.stream;
  const int64_t nsweeps = n - 2;
  const int64_t nJ = ceil_div(nsweeps, g);
  {
    const evd_status_t st = ensure_dynamic_smem((const void*)k_bcback_prep, smem);
    if (st != EVD_OK) return st;
  }
  auto kc = [&](int64_t J) { return sweep_steps_b(n, b, J * g); };
  const bool fused = pc.bcback_fused && pc.bb && bcback_fused_supported(pc, Q, ldq);
  if (identity && !fused) return EVD_ERR_INVALID_ARG;  // the identity start needs the fused waves
  if (fused) {
    evd_status_t st = bcback_fixed_point(pc, Q, ldq, true);
    if (st != EVD_OK) return st;
    st = fused_waves(pc, bw, Q, ldq, w, identity);
    if (st != EVD_OK) return st;
    return bcback_fixed_point(pc, Q, ldq, false);
  }
  const int64_t tmax = kc(0) + nJ - 2;
  for (int64_t t = 0; t <= tmax; ++t) {
    // groups of wave t: J' = nJ - 1 - J in [jlo, jhi] with 0 <= k = t - J' < kc(J)
    int64_t jp = std::min<int64_t>(t, nJ - 1);
    while (jp >= 0) {
      // skip invalid J' (descending), then take the maximal run of valid ones
      if (t - jp >= kc(nJ - 1 - jp)) { --jp; continue; }
      const int64_t jhi = jp;
      while (jp >= 0 && t - jp < kc(nJ - 1 - jp)) --jp;
      const int64_t jlo = jp + 1;
      const int count = (int)(jhi - jlo + 1);
      if ((size_t)count * h * g > w.vg_capacity || (size_t)count * n * g > w.wt_capacity)
        return ws_fail("bc_back wave buffers", w.wt_capacity, (size_t)count * n * g);
      {
        StatScope sc("bc_back_prep", s);
        k_bcback_prep<<<(unsigned)count, dim3(32, 8), smem, s>>>(bw.U, bw.Utau, n, b, g, nJ, t, jlo, w.Vg, w.Yg, h); count_launch();
        EVD_CUDA_TRY(cudaGetLastError());
      }
      // problem 0 (J' = jlo) is the lowest group of the run and the only one that may reach row n
      const int64_t J0 = nJ - 1 - jlo, k0 = t - jlo;
      const int64_t R0 = J0 * g + 1 + k0 * b;
      const int64_t hh0 = std::min<int64_t>(h, n - R0);
      Batch bt;
      bt.count = count;
      // W_p^T = X(R0_p : R0_p + h, :)^T V_p   (n x g each), R0_p = R0 - p (g + b)
      Gemm g1;
      g1.status = pc.status;
      g1.tag = "bc_back_gemm";
      g1.ta = 'T'; g1.m = n; g1.n = g; g1.k = h; g1.A = Q + R0; g1.lda = ldq; g1.B = w.Vg; g1.ldb = h;
      g1.C = w.Wt; g1.ldc = n; g1.alpha = 1.0; g1.beta = 0.0;
      bt.sA = -(int64_t)(g + b); bt.sB = (int64_t)h * g; bt.sC = n * g; bt.first_k = hh0; bt.first_m = -1;
      evd_status_t st = (count > 1) ? ozaki_gemm_batched(g1, bt, pc.slices, w.gemm_ws, w.gemm_ws_bytes, s)
                                    : (g1.k = hh0, gemm(g1, pc.slices, w.gemm_ws, w.gemm_ws_bytes, s));
      if (st != EVD_OK) return st;
      // X_p -= Y_p W_p
      Gemm g2;
      g2.status = pc.status;
      g2.tag = "bc_back_gemm";
      g2.tb = 'T'; g2.m = h; g2.n = n; g2.k = g; g2.A = w.Yg; g2.lda = h; g2.B = w.Wt; g2.ldb = n;
      g2.C = Q + R0; g2.ldc = ldq; g2.alpha = -1.0; g2.beta = 1.0;
      bt.sA = (int64_t)h * g; bt.sB = n * g; bt.sC = -(int64_t)(g + b); bt.first_k = -1; bt.first_m = hh0;
      st = (count > 1) ? ozaki_gemm_batched(g2, bt, pc.slices, w.gemm_ws, w.gemm_ws_bytes, s)
                       : (g2.m = hh0, gemm(g2, pc.slices, w.gemm_ws, w.gemm_ws_bytes, s));
      if (st != EVD_OK) return st;
    }
  }
  return EVD_OK;
}

// SBR-Back, blocked: Q_s = H_0 H_1 ... H_{np-1} with H_p = I - V_p T_p V_p^T.  Groups
// of kSbrBackPanels consecutive panels are merged into one compact WY form
// H_{p0} ... H_{p1} = I - V T V^T, V = [V_{p0} .. V_{p1}] (panel p's reflectors start
// (p - p0) b rows below the block's first row) and, panel by panel,
//     T = [[T_prev, -T_prev (V_prev^T V_p) T_p], [0, T_p]],
// so that X <- (I - V T V^T) X streams X once per group instead of once per panel.
// Groups are applied last group first, as the panels are.
evd_status_t sbr_back_run(const PlanCore& pc, const double* A, const double* sbr_T, const double* sbr_tau,
                          double* Q, int64_t ldq, const BackWork& w) {
  (void)sbr_tau;
  const int64_t n = pc.n, lda = pc.lda;
  const int b = pc.b;
  const int qmax = kSbrBackPanels;
  const int64_t ldk = (int64_t)qmax * b;  // leading dimension of the Kb x n buffers and of T_blk
  cudaStream_t s = pc.stream;
  int64_t np = 0;  // number of factored panels
  while (n - (np * b + b) >= 2) ++np;
  auto pgemm = [&](Gemm g, int slices) {
    g.status = pc.status;
    g.tag = "sbr_back";
    return gemm(g, slices, w.gemm_ws, w.gemm_ws_bytes, s);
  };
  for (int64_t p1 = np - 1; p1 >= 0; p1 -= qmax) {
    const int64_t p0 = std::max<int64_t>(0, p1 - qmax + 1);
    const int64_t R = p0 * b + b, M = n - R;  // rows of the block
    // explicit V of the block, and the width of each panel
    int kbs[kSbrBackPanels];
    int64_t Kb = 0;
    for (int64_t p = p0; p <= p1; ++p) {
      const int64_t c0 = p * b, r0 = c0 + b, m = n - r0;
      const int bw = (int)((n - c0 < b) ? n - c0 : b);
      const int kb = (int)((bw < m) ? bw : m);
      kbs[p - p0] = kb;
      k_explicit_v<<<dim3((unsigned)std::min<int64_t>(ceil_div(M, 256), 64), (unsigned)kb), 256, 0, s>>>(
          A, lda, r0, c0, (p - p0) * b, M, kb, w.Vp + Kb * n, n); count_launch();
      Kb += kb;
    }
    EVD_CUDA_TRY(cudaGetLastError());
    // T of the block (Kb x Kb, upper triangular, ld ldk)
    EVD_CUDA_TRY(cudaMemset2DAsync(w.Tblk, ldk * sizeof(double), 0, Kb * sizeof(double), Kb, s));
    int64_t Kp = 0;
    for (int64_t p = p0; p <= p1; ++p) {
      const int kb = kbs[p - p0];
      EVD_CUDA_TRY(cudaMemcpy2DAsync(w.Tblk + Kp + Kp * ldk, ldk * sizeof(double), sbr_T + (size_t)p * b * b,
                                     b * sizeof(double), kb * sizeof(double), kb, cudaMemcpyDeviceToDevice, s));
      if (Kp > 0) {
        // C = V_prev^T V_p   (Kp x kb, K = M)
        Gemm gc;
        gc.ta = 'T'; gc.m = Kp; gc.n = kb; gc.k = M; gc.A = w.Vp; gc.lda = n; gc.B = w.Vp + Kp * n; gc.ldb = n;
        gc.C = w.Cblk; gc.ldc = ldk; gc.alpha = 1.0; gc.beta = 0.0;
        evd_status_t st = pgemm(gc, pc.slices);
        if (st != EVD_OK) return st;
        // D = T_prev C, then T(0:Kp, Kp:Kp+kb) = -D T_p
        Gemm gd;
        gd.m = Kp; gd.n = kb; gd.k = Kp; gd.A = w.Tblk; gd.lda = ldk; gd.B = w.Cblk; gd.ldb = ldk;
        gd.C = w.Cblk + (size_t)ldk * b; gd.ldc = ldk; gd.alpha = 1.0; gd.beta = 0.0;
        st = pgemm(gd, pc.slices);  // the split product once Kp is large enough
        if (st != EVD_OK) return st;
        Gemm ge;
        ge.m = Kp; ge.n = kb; ge.k = kb; ge.A = gd.C; ge.lda = ldk; ge.B = w.Tblk + Kp + Kp * ldk; ge.ldb = ldk;
        ge.C = w.Tblk + Kp * ldk; ge.ldc = ldk; ge.alpha = -1.0; ge.beta = 0.0;
        st = pgemm(ge, 0);
        if (st != EVD_OK) return st;
      }
      Kp += kb;
    }
    // W = V^T X(R:, :)   (Kb x n)
    Gemm g1;
    g1.ta = 'T'; g1.m = Kb; g1.n = n; g1.k = M; g1.A = w.Vp; g1.lda = n; g1.B = Q + R; g1.ldb = ldq;
    g1.C = w.Wp; g1.ldc = ldk; g1.alpha = 1.0; g1.beta = 0.0;
    evd_status_t st = pgemm(g1, pc.slices);
    if (st != EVD_OK) return st;
    // Tp = T W  (Kb x n)
    Gemm g2;
    g2.m = Kb; g2.n = n; g2.k = Kb; g2.A = w.Tblk; g2.lda = ldk; g2.B = w.Wp; g2.ldb = ldk;
    g2.C = w.Tp; g2.ldc = ldk; g2.alpha = 1.0; g2.beta = 0.0;
    st = pgemm(g2, pc.slices);
    if (st != EVD_OK) return st;
    // X(R:, :) -= V Tp
    Gemm g3;
    g3.m = M; g3.n = n; g3.k = Kb; g3.A = w.Vp; g3.lda = n; g3.B = w.Tp; g3.ldb = ldk;
    g3.C = Q + R; g3.ldc = ldq; g3.alpha = -1.0; g3.beta = 1.0;
    st = pgemm(g3, pc.slices);
    if (st != EVD_OK) return st;
  }
  return EVD_OK;
}

}  // namespace evd
