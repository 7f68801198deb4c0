// FP64-accurate dense products on the tcgen05 tensor cores (sm_103a).
//
// The FP64 operands are split into s bfloat16 slices (Ozaki-style error-free
// splitting with balanced base-2^7 digits, after a power-of-two scaling of every row
// of the left operand and every column of the right operand):
//     a_rk = 2^(e_r) sum_t sigma_t 2^(-7 (t+1)),  |sigma_0| <= 128, |sigma_t| <= 64.
// A digit is an integer of at most 8 significant bits, so it is exact in bfloat16;
// a product of two digits is exact in FP32.  The kernel forms, for every weight
// k = t + u <= s-1, S_k = sum over pairs (t, u) and over K of sigma^A_t sigma^B_u with
// tcgen05.mma kind::f16 into an FP32 accumulator in tensor memory (64 columns per
// weight, weight k at columns 64 k).  One instruction multiplies slice t of A by
// up to four consecutive slices u0..u0+3 of B stacked along N (N <= 256), which
// lands in the accumulators of weights t+u0..t+u0+3 -- 12 instructions per K-step
// instead of 36.  The accumulators are drained every 384 K-elements; a weight-k
// accumulator then never exceeds (k+3) 2^12 * 384 < 2^24 in magnitude (k <= 7),
// so every partial sum is an exact integer; drains are converted to int64 and
// combined exactly, with left shifts only, into two accumulators
//     R_hi = sum_{k <= H} S_k 2^(7 (H - k))      H = min(s-1, 3)
//     R_lo = sum_{4 <= k <= s-1} S_k 2^(7 (s-1-k))
// (both stay below 2^53 for K <= 2^17), and finally
// C = alpha (2^(e_r + f_c - 14 - 7H) R_hi + 2^(e_r + f_c - 14 - 7(s-1)) R_lo) + beta C
// in FP64.
//
// Slice layout ("blobs"): the split kernels write each operand as blobs, one per
// (row tile, K-block of 16): s slices x TR rows x 16 K-elements (TR = 128 for the
// left operand, 64 for the right), each slice in the tensor core's canonical
// K-major layout without swizzle -- core matrices of 8 rows x 8 elements (128 bytes)
// ordered (row group, K half).  A stage of the product is then one contiguous bulk
// copy per operand (s x 4 KB and s x 2 KB) instead of a box of 32-byte rows.
//
// Kernel structure (one CTA per 128 x 64 tile of C, 320 threads):
//   warp 0      copy producer: one bulk copy per operand and stage, 4 stages.
//   warp 1      tensor-memory allocation (512 columns) and the single MMA-issuing
//               thread: per stage, every slice pair (t, u) with t + u <= s-1.
//   warps 2..9  epilogue: drains all weight accumulators every 16 stages into
//               int64 registers, then the FP64 write of C.
// Every mbarrier wait is bounded; on timeout the CTA raises the abort flag, sets
// EVD_ERR_TIMEOUT in the status word and leaves after freeing tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "device_util.cuh"
#include "evd_ozaki.h"
#include "tc_common.cuh"

namespace evd {

namespace {

using namespace tcx;

constexpr int OZ_STAGES = 4;
constexpr int OZ_THREADS = 320;
constexpr int OZ_PERIOD = 24;     // stages between two drains of one weight (384 K-elements)
constexpr int OZ_GROUP_M = 8;     // row tiles per rasterization group
constexpr uint32_t OZ_PARK_BYTES = 256 * 64 * 8;  // epilogue: 2 x 32 int64 sums per epilogue thread

// ------------------------------------------------------------------ operand views
// Element (rho, kappa) of an operand seen as rows x K:
//   mode 0: p[rho + kappa ld]   mode 1: p[kappa + rho ld]
//   mode 2: symmetric, lower triangle stored: p[max + min ld]
struct View {
  const double* p;
  int64_t ld;
  int mode;
  int64_t rows, K;
  int64_t pstride = 0;  // batched: element offset between consecutive problems
  int64_t K0 = -1;      // batched: K of problem 0 when >= 0 (a truncated first problem)
  int64_t koff = 0;     // K-elements 0 .. koff-1 are zero, K-element kappa >= koff is p's kappa - koff
  __device__ __forceinline__ double get(int64_t r, int64_t k) const {
    if (mode == 0) return p[r + k * ld];
    if (mode == 1) return p[k + r * ld];
    return (r >= k) ? p[r + k * ld] : p[k + r * ld];
  }
  __device__ __forceinline__ bool row_contig() const { return mode != 1; }
};

__device__ __forceinline__ void load_tile32(const View& v, int64_t r0, int64_t k0, double (*t)[33]) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int idx = tid; idx < 1024; idx += 256) {
    const int a = idx & 31, b = idx >> 5;
    const int r = v.row_contig() ? a : b, k = v.row_contig() ? b : a;
    const int64_t R = r0 + r, KK = k0 + k;
    t[r][k] = (R < v.rows && KK < v.K && KK >= v.koff) ? v.get(R, KK - v.koff) : 0.0;
  }
}

// Max biased exponent of each row, atomicMax into ex[] (pre-zeroed).
__global__ void k_row_exponent(const View v, int* ex, int64_t kspan) {
  __shared__ double t[32][33];
  __shared__ int red[8][32];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int64_t kb = (int64_t)blockIdx.y * kspan;
  int mx = 0;
  for (int64_t k0 = kb; k0 < kb + kspan && k0 < v.K; k0 += 32) {
    __syncthreads();
    load_tile32(v, r0, k0, t);
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
      const unsigned long long bits = (unsigned long long)__double_as_longlong(t[threadIdx.x][k]);
      mx = max(mx, (int)((bits >> 52) & 0x7FF));
    }
  }
  red[threadIdx.y][threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.y == 0) {
    for (int y = 1; y < 8; ++y) mx = max(mx, red[y][threadIdx.x]);
    if (r0 + threadIdx.x < v.rows && mx > 0) atomicMax(ex + r0 + threadIdx.x, mx);
  }
}

// Slices S[t][rho][kappa] (bfloat16, K-major, rows_pad x K_pad per slice) and the
// frexp exponent per row (ex holds the max biased exponent on entry).
__global__ void k_split(const View v, const int* ex_biased, int* ex_frexp, int s, int64_t rows_pad, int64_t K_pad,
                        __nv_bfloat16* S, int TR) {
  __shared__ double t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  load_tile32(v, r0, k0, t);
  __syncthreads();
  const int tid = threadIdx.y * 32 + threadIdx.x;
  // each thread: row r = tid / 16 + 16 j, kappa pair (2 q, 2 q + 1) with q = tid % 16
  const int q = tid & 15;
  for (int rr = tid >> 4; rr < 32; rr += 16) {
    const int64_t R = r0 + rr;
    int eb = (R < v.rows) ? ex_biased[R] : 0;
    const int e = (eb > 0) ? eb - 1022 : -1022;
    if (k0 == 0 && q == 0 && R < rows_pad) ex_frexp[R] = e;
    const long long off = ozaki_offset(s);
    const long long T0 = ozaki_scaled(t[rr][2 * q], e, s) + off;
    const long long T1 = ozaki_scaled(t[rr][2 * q + 1], e, s) + off;
    const int64_t nkb = K_pad / 16;
    for (int tt = 0; tt < s; ++tt) {
      __nv_bfloat162 h;
      h.x = __float2bfloat16_rn((float)ozaki_digit(T0, s, tt));
      h.y = __float2bfloat16_rn((float)ozaki_digit(T1, s, tt));
      *reinterpret_cast<__nv_bfloat162*>(S + blob_index(R, k0 + 2 * q, tt, s, TR, nkb)) = h;
    }
  }
}

// One-pass split for short K (K_pad <= 512) of both operands in one launch: block
// x < nblk_a takes 32 rows of A, the others 32 rows of B.  The block caches its
// 32 x K_pad rows in shared memory (all loads issued up front), reduces the row
// exponents, then writes the digits 8 K-elements (16 bytes) per slice at a time.
__global__ void __launch_bounds__(256) k_split_fused(const View va, int* ea, __nv_bfloat16* SA, int64_t rows_pad_a,
                                                     const View vb, int* eb, __nv_bfloat16* SB, int64_t rows_pad_b,
                                                     int nblk_a, int s, int64_t K_pad) {
  extern __shared__ double tile[];  // [32][K_pad + 1]
  const bool isA = (int)blockIdx.x < nblk_a;
  View v = isA ? va : vb;
  // batched: problem p = blockIdx.y; slices S[t][p rows_pad + r][K_pad], exponents ex[p rows_pad + r]
  const int64_t pb = blockIdx.y, count = gridDim.y;
  v.p += pb * v.pstride;
  if (pb == 0 && v.K0 >= 0) v.K = v.K0;
  const int64_t rows_pad = isA ? rows_pad_a : rows_pad_b;
  int* ex = (isA ? ea : eb) + pb * rows_pad;
  __nv_bfloat16* S = isA ? SA : SB;
  const int TR = isA ? 128 : 64;
  const int64_t nkb = K_pad / 16;
  (void)count;
  const int64_t r0 = (int64_t)(isA ? (int)blockIdx.x : (int)blockIdx.x - nblk_a) * 32;
  const int ls = (int)K_pad + 1;
  const int tid = threadIdx.x;
  const int total = 32 * (int)K_pad;
  if (v.row_contig()) {
#pragma unroll 8
    for (int idx = tid; idx < total; idx += 256) {
      const int r = idx & 31, k = idx >> 5;
      const int64_t R = r0 + r;
      tile[r * ls + k] = (R < v.rows && k < v.K && k >= v.koff) ? v.get(R, k - v.koff) : 0.0;
    }
  } else {
#pragma unroll 8
    for (int idx = tid; idx < total; idx += 256) {
      const int t2 = idx >> 5;
      const int r = t2 & 31, k = ((t2 >> 5) << 5) + (idx & 31);
      const int64_t R = r0 + r;
      tile[r * ls + k] = (R < v.rows && k < v.K && k >= v.koff) ? v.get(R, k - v.koff) : 0.0;
    }
  }
  __syncthreads();
  // row r = tid / 8: max biased exponent over its K range, 8 threads per row
  const int r = tid >> 3, q = tid & 7;
  int mx = 0;
  for (int k = q; k < (int)K_pad; k += 8)
    mx = max(mx, (int)((__double_as_longlong(tile[r * ls + k]) >> 52) & 0x7FF));
  mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
  mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
  const int e = (mx > 0) ? mx - 1022 : -1022;
  const int64_t R = r0 + r;
  if (q == 0) ex[R] = e;
  // digits: units of 8 K-elements, unit u = q + 8 j
  for (int u = q; u < (int)K_pad / 8; u += 8) {
    const long long off = ozaki_offset(s);
    long long TO[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) TO[i] = ozaki_scaled(tile[r * ls + 8 * u + i], e, s) + off;
    for (int tt = 0; tt < s; ++tt) {
      uint32_t w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h;
        h.x = __float2bfloat16_rn((float)ozaki_digit(TO[2 * i], s, tt));
        h.y = __float2bfloat16_rn((float)ozaki_digit(TO[2 * i + 1], s, tt));
        w[i] = *reinterpret_cast<uint32_t*>(&h);
      }
      *reinterpret_cast<uint4*>(S + blob_index(pb * rows_pad + R, 8 * u, tt, s, TR, nkb)) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

struct MmaArgs {
  const __nv_bfloat16* SA;  // left operand blobs
  const __nv_bfloat16* SB;  // right operand blobs
  int64_t nkb;              // K-blocks of 16 per row tile
  int64_t m, n;
  int s;            // slices
  int nst;          // stages = K_pad / OZ_KS
  uint32_t tmem_cols;
  const int* ea;    // frexp exponents of the rows of the left operand
  const int* eb;    // ... of the columns of the right operand
  double* C;
  int64_t ldc;
  double alpha, beta;
  int lower;
  int* st;
  int stages_per_split;  // split K: CTA z handles stages [z * stages_per_split, ...)
  double* part;          // split K: partial products (alpha = 1, beta = 0), m x n each, ld m
  // batched (grid z = problem): problem p reads slice rows p bm_pad + ... of A and
  // p bn_pad + ... of B and writes C + p sC; problem 0 writes only m_first rows
  int batched;
  int64_t bm_pad, bn_pad, sC, m_first;
  int64_t nkb_b;   // K-blocks per row tile of B's blob (A's is nkb)
  int64_t c_skip;  // the first c_skip rows of the product are not stored; row r goes to row r - c_skip of C
};

__device__ __forceinline__ bool drain_after(int j, int nst) {
  return (j % OZ_PERIOD == OZ_PERIOD - 1) || (j == nst - 1);
}

template <int S>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_ozaki_mma(const MmaArgs a) {
  extern __shared__ uint8_t smem_raw[];
  // grouped rasterization: consecutive CTAs sweep OZ_GROUP_M row tiles for each
  // column tile, so a wave shares both operands' slices in L2
  const int num_m = (int)gridDim.x, num_n = (int)gridDim.y;
  const int id = (int)(blockIdx.x + (int64_t)blockIdx.y * gridDim.x);
  const int group = id / (OZ_GROUP_M * num_n);
  const int first_m = group * OZ_GROUP_M;
  const int gm = (num_m - first_m < OZ_GROUP_M) ? num_m - first_m : OZ_GROUP_M;
  const int in_group = id - group * OZ_GROUP_M * num_n;
  const int mt = first_m + in_group % gm, nt = in_group / gm;
  const int64_t m0 = (int64_t)mt * OZ_BM, n0 = (int64_t)nt * OZ_BN;
  if (a.lower && n0 > m0 + OZ_BM - 1) return;  // tile strictly above the diagonal
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int s = S, L = S - 1;
  const int64_t pb = a.batched ? (int64_t)blockIdx.z : 0;
  const int j0 = a.batched ? 0 : (int)blockIdx.z * a.stages_per_split;
  const int nst = (a.nst - j0 < a.stages_per_split) ? a.nst - j0 : a.stages_per_split;
  // blobs of this CTA's row tiles: stage j reads K-block j0 + j
  const __nv_bfloat16* blobA = a.SA + (size_t)((pb * a.bm_pad + m0) / OZ_BM) * a.nkb * s * (OZ_BM * OZ_KS);
  const __nv_bfloat16* blobB = a.SB + (size_t)((pb * a.bn_pad + n0) / OZ_BN) * a.nkb_b * s * (OZ_BN * OZ_KS);
  const int* ea = a.ea + pb * a.bm_pad;
  const int* eb = a.eb + pb * a.bn_pad;
  double* Cp = a.C + pb * a.sC;
  const int64_t m_lim = (pb == 0 && a.m_first >= 0) ? a.m_first : a.m;
  const uint32_t a_bytes = (uint32_t)s * OZ_BM * OZ_KS * 2, b_bytes = (uint32_t)s * OZ_BN * OZ_KS * 2;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const uint32_t data_bytes = (OZ_STAGES * stage_bytes > OZ_PARK_BYTES) ? OZ_STAGES * stage_bytes : OZ_PARK_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + data_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + OZ_STAGES;
  uint64_t* accf = bars + 2 * OZ_STAGES;
  uint64_t* acce = bars + 2 * OZ_STAGES + OZ_MAXS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * OZ_STAGES + 2 * OZ_MAXS);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* eb_s = reinterpret_cast<int*>(tmem_slot + 4);  // column exponents of this tile (OZ_BN ints)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < OZ_STAGES; ++i) { mbar_init(smem_u32(full + i), 1); mbar_init(smem_u32(empty + i), 1); }
    mbar_init(smem_u32(accf), 1);
    mbar_init(smem_u32(acce), 8);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int issued = 0;
      for (int j = 0; j < nst; ++j) {
        const int si = j % OZ_STAGES, round = j / OZ_STAGES;
        if (round > 0 && !mbar_wait(smem_u32(empty + si), (round - 1) & 1, abort, a.st, 9001)) break;
        uint8_t* sa = smem + si * stage_bytes;
        const uint32_t fb = smem_u32(full + si);
        mbar_expect_tx(fb, stage_bytes);
        bulk_load(smem_u32(sa), blobA + (size_t)(j0 + j) * s * (OZ_BM * OZ_KS), a_bytes, fb);
        bulk_load(smem_u32(sa + a_bytes), blobB + (size_t)(j0 + j) * s * (OZ_BN * OZ_KS), b_bytes, fb);
        ++issued;
      }
      if (*abort) {
        // let the copies already in flight land before the CTA exits
        for (int j = (issued > OZ_STAGES ? issued - OZ_STAGES : 0); j < issued; ++j) {
          const int si = j % OZ_STAGES, round = j / OZ_STAGES;
          for (long long i = 0; i < OZ_WAIT_LIMIT && !mbar_try(smem_u32(full + si), round & 1); ++i) {}
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int chunk = 0;
      const uint64_t da_base = desc_kmajor(smem_u32(smem));
      for (int j = 0; j < nst && !*abort; ++j) {
        const int si = j % OZ_STAGES, round = j / OZ_STAGES;
        if (!mbar_wait(smem_u32(full + si), round & 1, abort, a.st, 9002)) break;
        tc_fence_after();
        const bool fresh = (j % OZ_PERIOD) == 0;
        if (fresh && j > 0) {
          if (!mbar_wait(smem_u32(acce), (chunk - 1) & 1, abort, a.st, 9003)) break;
          tc_fence_after();
        }
        const uint64_t da0 = da_base + (uint64_t)((si * stage_bytes) >> 4);
        const uint64_t db0 = da0 + (uint64_t)(a_bytes >> 4);
        issue_stage<S>(tmem, da0, db0, fresh ? 0u : 1u);
        if (drain_after(j, nst)) {
          tc_commit(smem_u32(accf));
          ++chunk;
        }
        tc_commit(smem_u32(empty + si));
      }
    }
  } else {
    // ---------------- epilogue warps 2..9
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const int64_t row = m0 + quad * 32 + lane;
    const int H = (L < 3) ? L : 3;
    // exponents first, while the main loop runs: the row's in a register, the
    // tile's columns in shared memory (named barrier over the 8 epilogue warps)
    const int etid = threadIdx.x - 64;
    if (etid < OZ_BN) eb_s[etid] = (n0 + etid < a.n) ? eb[n0 + etid] : 0;
    const int er = (row < a.m) ? ea[row] : 0;
    asm volatile("bar.sync 1, 256;" ::: "memory");
    long long Rh[32], Rl[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) { Rh[c] = 0; Rl[c] = 0; }
    bool ok = true;
    int chunk = 0;
    for (int j = 0; j < nst && ok; ++j) {
      if (!drain_after(j, nst)) continue;
      if (!mbar_wait(smem_u32(accf), chunk & 1, abort, a.st, 9004)) { ok = false; break; }
      ++chunk;
      tc_fence_after();
      for (int k = 0; k <= L; ++k) {
        const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(k * OZ_BN + half * 32);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v[16];
          tc_ld16(taddr + 16 * h, v);
          if (k <= 3) {
            const int sh = 7 * (H - k);
#pragma unroll
            for (int c = 0; c < 16; ++c) Rh[16 * h + c] += (long long)__float2int_rn(v[c]) << sh;
          } else {
            const int sh = 7 * (L - k);
#pragma unroll
            for (int c = 0; c < 16; ++c) Rl[16 * h + c] += (long long)__float2int_rn(v[c]) << sh;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(acce));
    }
    if (ok) {
      // Every MMA has retired (last accumulator barrier) and every TMA load has
      // landed, so the stage buffers are idle: park the exact sums there and let a
      // rolled loop index them.  The output code runs once per CTA, and a fully
      // unrolled version of it would be fetched cold from L2.
      long long* park = reinterpret_cast<long long*>(smem) + (threadIdx.x - 64);  // [2 * 32][256]
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        park[(2 * c) * 256] = Rh[c];
        park[(2 * c + 1) * 256] = Rl[c];
      }
      if (row >= a.c_skip && row < m_lim) {
        const int shift_hi = 7 * (L - H);  // R = R_hi 2^(7 (L - H)) + R_lo, value R 2^(e_r + f_c - 14 - 7L)
        const bool alpha_one = (a.alpha == 1.0), alpha_mone = (a.alpha == -1.0);
        const bool read_c = (a.part == nullptr) && (a.beta != 0.0);
        double* crow = Cp + (row - a.c_skip);
        const int64_t mo = a.m - a.c_skip;  // stored rows
#pragma unroll 1
        for (int c0 = 0; c0 < 32; c0 += 4) {
          // the 4 loads of C go out before any store so that they overlap
          double cv[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int64_t col = n0 + half * 32 + c0 + c;
            const bool valid = col < a.n && !(a.lower && row < col);
            cv[c] = (read_c && valid) ? crow[col * a.ldc] : 0.0;
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int cc = c0 + c;
            const int64_t col = n0 + half * 32 + cc;
            if (col < a.n && !(a.lower && row < col)) {
              // exact 128-bit R = Rh << shift_hi + Rl
              const long long rh = park[(2 * cc) * 256];
              unsigned long long lo = (shift_hi == 0) ? (unsigned long long)rh : ((unsigned long long)rh << shift_hi);
              long long hi = (shift_hi == 0) ? (rh >> 63) : (rh >> (64 - shift_hi));
              if (L >= 4) {
                const long long rl = park[(2 * cc + 1) * 256];
                const unsigned long long nlo = lo + (unsigned long long)rl;
                hi += (rl >> 63) + (nlo < lo ? 1 : 0);
                lo = nlo;
              }
              double v = i128_to_double(hi, lo, er + eb_s[half * 32 + cc] - 14 - 7 * L);
              if (a.part) {
                a.part[(size_t)blockIdx.z * mo * a.n + (row - a.c_skip) + col * mo] = v;
              } else {
                if (alpha_mone) v = -v;
                else if (!alpha_one) v *= a.alpha;
                if (read_c) v = (a.beta == 1.0) ? (cv[c] + v) : fma(a.beta, cv[c], v);
                crow[col * a.ldc] = v;
              }
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

// C = alpha sum_z part_z + beta C (split K), fixed summation order.
__global__ void k_splitk_reduce(const double* part, int splits, int64_t m, int64_t n, double alpha, double beta,
                                double* C, int64_t ldc, int lower) {
  const int64_t j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (lower && i < j) continue;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[(size_t)z * m * n + i + j * m];
    double* p = C + i + j * ldc;
    double v = alpha * s;
    if (beta != 0.0) v = fma(beta, *p, v);
    *p = v;
  }
}

// ------------------------------------------------------------------ host side
const void* mma_kernel(int slices) {
  switch (slices) {
    case 1: return (const void*)k_ozaki_mma<1>;
    case 2: return (const void*)k_ozaki_mma<2>;
    case 3: return (const void*)k_ozaki_mma<3>;
    case 4: return (const void*)k_ozaki_mma<4>;
    case 5: return (const void*)k_ozaki_mma<5>;
    case 6: return (const void*)k_ozaki_mma<6>;
    case 7: return (const void*)k_ozaki_mma<7>;
    default: return (const void*)k_ozaki_mma<8>;
  }
}
struct Pads {
  int64_t m_pad, n_pad, k_pad;
};
Pads pads(int64_t m, int64_t n, int64_t k) {
  return {ceil_div(m, OZ_BM) * OZ_BM, ceil_div(n, OZ_BN) * OZ_BN, ceil_div(k, 32) * 32};
}

// split K when the tile grid cannot fill the GPU: returns the split count
int splitk_count(int64_t m, int64_t n, int64_t k) {
  const int64_t tiles = ceil_div(m, OZ_BM) * ceil_div(n, OZ_BN);
  const int64_t k_pad = ceil_div(k, 32) * 32;
  int sms = 152;
  if (tiles >= sms || k_pad < 1024) return 1;
  int64_t sp = ceil_div(sms, tiles);
  sp = std::min<int64_t>(sp, k_pad / 512);
  if (m * n * sp > ((int64_t)1 << 27)) sp = std::max<int64_t>(1, ((int64_t)1 << 27) / (m * n));
  return (int)std::max<int64_t>(sp, 1);
}

// status word for timeouts of stand-alone products (allocated once)
int* standalone_status() {
  static int* d = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    if (cudaMalloc(&d, sizeof(int) * kStatusWords) == cudaSuccess) cudaMemset(d, 0, sizeof(int) * kStatusWords);
    else d = nullptr;
  });
  return d;
}

size_t smem_bytes(int s) {
  const size_t stages = (size_t)OZ_STAGES * s * (OZ_BM + OZ_BN) * OZ_KS * 2;
  return 1024 + std::max<size_t>(stages, OZ_PARK_BYTES) + (2 * OZ_STAGES + 2 * OZ_MAXS) * 8 + 16 + OZ_BN * 4;
}

}  // namespace

// Scratch of a (batched) product with `splits` K-splits (partials only when > 1).
size_t scratch_with_splits(int64_t m, int64_t n, int64_t k, int slices, int count, int splits) {
  if (slices <= 0 || count <= 0) return 0;
  Pads p = pads(m, n, k);
  Carver c(nullptr);
  c.take<__nv_bfloat16>((size_t)slices * count * p.m_pad * p.k_pad);
  c.take<__nv_bfloat16>((size_t)slices * count * p.n_pad * p.k_pad);
  c.take<int>((size_t)p.m_pad);
  c.take<int>((size_t)p.n_pad);
  c.take<int>((size_t)count * p.m_pad);
  c.take<int>((size_t)count * p.n_pad);
  c.take<double>(splits > 1 ? (size_t)splits * m * n : 0);
  return c.off + 256;
}

// The scratch a product prefers (with its preferred K-split count).  A smaller
// scratch down to the no-split size also works: the split count is then lowered.
size_t ozaki_scratch_bytes_batched(int64_t m, int64_t n, int64_t k, int slices, int count) {
  return scratch_with_splits(m, n, k, slices, count, count == 1 ? splitk_count(m, n, k) : 1);
}

size_t ozaki_scratch_bytes(int64_t m, int64_t n, int64_t k, int slices) {
  return ozaki_scratch_bytes_batched(m, n, k, slices, 1);
}

size_t ozaki_scratch_bytes_min(int64_t m, int64_t n, int64_t k, int slices) {
  return scratch_with_splits(m, n, k, slices, 1, 1);
}

evd_status_t standalone_status_take(int* code, int* info) {
  *code = 0;
  *info = 0;
  int* d = standalone_status();
  if (!d) return EVD_OK;  // never allocated: no stand-alone product has run
  int h[kStatusWords] = {0};
  EVD_CUDA_TRY(cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost));
  EVD_CUDA_TRY(cudaMemset(d, 0, sizeof(h)));
  *code = h[0];
  *info = h[1];
  return EVD_OK;
}

// Products from about 2 x 256 x 256 x 128 flops up run on the tensor cores: GB300's
// FP64 CUDA cores (about 1.1 TFLOP/s for the whole GPU) make even thin products with
// a long K slower there than the split product's few launches.
bool ozaki_eligible(const Gemm& g) {
  if (g.k < 32 || g.m < 16 || g.n < 16) return false;
  if (g.m > (int64_t)1 << 30 || g.n > (int64_t)1 << 30 || g.k > ((int64_t)1 << 17)) return false;
  return 2.0 * (double)g.m * (double)g.n * (double)g.k >= 1.6e7;
}

evd_status_t ozaki_gemm_batched(const Gemm& g, const Batch& bt, int slices, void* scratch, size_t scratch_bytes,
                                cudaStream_t s) {
  if (slices < 1 || slices > OZ_MAXS) return EVD_ERR_INVALID_ARG;
  const int count = bt.count;
  if (count < 1 || count > 65535) return EVD_ERR_INVALID_ARG;
  if (count > 1 && (g.lower || g.a_sym_lower)) return EVD_ERR_INVALID_ARG;
  if (!scratch || scratch_bytes < scratch_with_splits(g.m, g.n, g.k, slices, count, 1))
    return ws_fail(g.tag ? g.tag : "split product", scratch_bytes, scratch_with_splits(g.m, g.n, g.k, slices, count, 1));
  if (g.k > ((int64_t)1 << 17)) return EVD_ERR_NOT_SUPPORTED;  // exactness bound of the int64 sums
  const Pads p = pads(g.m, g.n, g.k);
  if (count > 1 && p.k_pad > 512) return EVD_ERR_NOT_SUPPORTED;  // batched products use the one-pass split
  if ((int64_t)count * std::max(p.m_pad, p.n_pad) > ((int64_t)1 << 31) - 1) return EVD_ERR_NOT_SUPPORTED;
  Carver c(scratch);
  __nv_bfloat16* SA = c.take<__nv_bfloat16>((size_t)slices * count * p.m_pad * p.k_pad);
  __nv_bfloat16* SB = c.take<__nv_bfloat16>((size_t)slices * count * p.n_pad * p.k_pad);
  int* exA = c.take<int>((size_t)p.m_pad);
  int* exB = c.take<int>((size_t)p.n_pad);
  int* eA = c.take<int>((size_t)count * p.m_pad);
  int* eB = c.take<int>((size_t)count * p.n_pad);
  int splits = (count == 1) ? splitk_count(g.m, g.n, g.k) : 1;
  while (splits > 1 && scratch_with_splits(g.m, g.n, g.k, slices, count, splits) > scratch_bytes) --splits;
  double* part = c.take<double>(splits > 1 ? (size_t)splits * g.m * g.n : 0);
  View va, vb;
  va.p = g.A; va.ld = g.lda; va.rows = g.m; va.K = g.k;
  va.mode = g.a_sym_lower ? 2 : (g.ta == 'N' ? 0 : 1);
  va.pstride = bt.sA; va.K0 = (count > 1 && bt.first_k >= 0) ? std::min<int64_t>(bt.first_k, g.k) : -1;
  vb.p = g.B; vb.ld = g.ldb; vb.rows = g.n; vb.K = g.k;
  vb.mode = (g.tb == 'N') ? 1 : 0;
  vb.pstride = bt.sB;
  const double flops = (double)count * (g.lower ? 1.0 : 2.0) * (double)g.m * (double)g.n * (double)g.k;
  {
    StatScope sc(g.tag ? g.tag : "gemm", s, 0.0,
                 (double)count * (8.0 * (double)(g.m + g.n) * (double)g.k * 2.0 +
                                  2.0 * slices * (double)(p.m_pad + p.n_pad) * p.k_pad), "tc_split_prep");
    dim3 blk(32, 8);
    if (p.k_pad <= 512) {
      {
        const evd_status_t st = ensure_dynamic_smem((const void*)k_split_fused, 32 * (512 + 1) * sizeof(double));
        if (st != EVD_OK) return st;
      }
      const int nblk_a = (int)(p.m_pad / 32), nblk_b = (int)(p.n_pad / 32);
      k_split_fused<<<dim3((unsigned)(nblk_a + nblk_b), (unsigned)count), 256, 32 * (p.k_pad + 1) * sizeof(double),
                      s>>>(va, eA, SA, p.m_pad, vb, eB, SB, p.n_pad, nblk_a, slices, p.k_pad); count_launch();
    } else {
      EVD_CUDA_TRY(cudaMemsetAsync(exA, 0, sizeof(int) * p.m_pad, s));
      EVD_CUDA_TRY(cudaMemsetAsync(exB, 0, sizeof(int) * p.n_pad, s));
      const int64_t kspan = 1024;
      k_row_exponent<<<dim3((unsigned)ceil_div(g.m, 32), (unsigned)ceil_div(g.k, kspan)), blk, 0, s>>>(va, exA, kspan); count_launch();
      k_row_exponent<<<dim3((unsigned)ceil_div(g.n, 32), (unsigned)ceil_div(g.k, kspan)), blk, 0, s>>>(vb, exB, kspan); count_launch();
      k_split<<<dim3((unsigned)(p.m_pad / 32), (unsigned)(p.k_pad / 32)), blk, 0, s>>>(va, exA, eA, slices, p.m_pad,
                                                                                     p.k_pad, SA, OZ_BM); count_launch();
      k_split<<<dim3((unsigned)(p.n_pad / 32), (unsigned)(p.k_pad / 32)), blk, 0, s>>>(vb, exB, eB, slices, p.n_pad,
                                                                                     p.k_pad, SB, OZ_BN); count_launch();
    }
    EVD_CUDA_TRY(cudaGetLastError());
  }
  MmaArgs a;
  a.SA = SA; a.SB = SB; a.nkb = p.k_pad / OZ_KS; a.nkb_b = a.nkb; a.c_skip = 0;
  a.m = g.m; a.n = g.n; a.s = slices; a.nst = (int)(p.k_pad / OZ_KS);
  uint32_t cols = 64;
  while (cols < (uint32_t)(slices * OZ_BN)) cols <<= 1;
  a.tmem_cols = cols;
  a.ea = eA; a.eb = eB; a.C = g.C; a.ldc = g.ldc; a.alpha = g.alpha; a.beta = g.beta;
  a.lower = g.lower ? 1 : 0; a.st = nullptr;
  a.batched = (count > 1) ? 1 : 0;
  a.bm_pad = p.m_pad; a.bn_pad = p.n_pad; a.sC = bt.sC;
  a.m_first = (count > 1 && bt.first_m >= 0) ? std::min<int64_t>(bt.first_m, g.m) : -1;
  {
    // stages per split: a multiple of the drain period so chunks stay aligned
    const int per = (int)ceil_div(ceil_div(a.nst, splits), OZ_PERIOD) * OZ_PERIOD;
    a.stages_per_split = per;
  }
  const int zsplits = (int)ceil_div(a.nst, a.stages_per_split);
  a.part = (zsplits > 1) ? part : nullptr;
  a.st = g.status ? g.status : standalone_status();
  if (!a.st) return EVD_ERR_OOM;
  const size_t smem = smem_bytes(slices);
  {
    const evd_status_t st = ensure_dynamic_smem(mma_kernel(slices), smem_bytes(OZ_MAXS));
    if (st != EVD_OK) return st;
  }
  dim3 grid((unsigned)(p.m_pad / OZ_BM), (unsigned)(p.n_pad / OZ_BN), (unsigned)(count > 1 ? count : zsplits));
  if (grid.y > 65535) return EVD_ERR_INVALID_ARG;
  StatScope sc(g.tag ? g.tag : "gemm", s, flops * (double)(slices * (slices + 1) / 2), 0.0, "tc_split");
  void* kargs[] = {&a};
  EVD_CUDA_TRY(cudaLaunchKernel(mma_kernel(slices), grid, dim3(OZ_THREADS), kargs, smem, s)); count_launch();
  EVD_CUDA_TRY(cudaGetLastError());
  if (zsplits > 1) {
    for (int64_t j0 = 0; j0 < g.n; j0 += 65535) {
      const int64_t cols = std::min<int64_t>(g.n - j0, 65535);
      k_splitk_reduce<<<dim3((unsigned)std::min<int64_t>(ceil_div(g.m, 256), 16), (unsigned)cols), 256, 0, s>>>(
          part + j0 * g.m, zsplits, g.m, g.n, g.alpha, g.beta, g.C + j0 * g.ldc, g.ldc, g.lower ? 1 : 0); count_launch();
    }
    EVD_CUDA_TRY(cudaGetLastError());
  }
  return EVD_OK;
}

evd_status_t ozaki_gemm(const Gemm& g, int slices, void* scratch, size_t scratch_bytes, cudaStream_t s) {
  return ozaki_gemm_batched(g, Batch(), slices, scratch, scratch_bytes, s);
}

// ------------------------------------------------------------------ presplit operand
size_t ozaki_presplit_bytes(int64_t m, int slices) {
  const Pads p = pads(m, OZ_BN, m);
  Carver c(nullptr);
  c.take<__nv_bfloat16>((size_t)slices * p.m_pad * p.k_pad);
  c.take<int>((size_t)p.m_pad);
  c.take<int>((size_t)p.m_pad);
  return c.off + 256;
}

evd_status_t ozaki_presplit_sym(const double* A, int64_t lda, int64_t m, int slices, void* buf, size_t bytes,
                                const char* tag, SplitOperand* out, cudaStream_t s) {
  if (slices < 1 || slices > OZ_MAXS || m < 1 || m > ((int64_t)1 << 17) || !out) return EVD_ERR_INVALID_ARG;
  if (!buf || bytes < ozaki_presplit_bytes(m, slices)) return ws_fail(tag, bytes, ozaki_presplit_bytes(m, slices));
  const Pads p = pads(m, OZ_BN, m);
  Carver c(buf);
  SplitOperand o;
  o.S = c.take<__nv_bfloat16>((size_t)slices * p.m_pad * p.k_pad);
  int* exb = c.take<int>((size_t)p.m_pad);
  o.e = c.take<int>((size_t)p.m_pad);
  o.rows = m; o.rows_pad = p.m_pad; o.K_pad = p.k_pad; o.slices = slices;
  o.bytes = c.off + 256;
  View va;
  va.p = A; va.ld = lda; va.rows = m; va.K = m; va.mode = 2;
  {
    StatScope sc(tag, s, 0.0, 8.0 * (double)m * (double)m * 2.0 + 2.0 * slices * (double)p.m_pad * p.k_pad,
                 "tc_split_prep");
    EVD_CUDA_TRY(cudaMemsetAsync(exb, 0, sizeof(int) * p.m_pad, s));
    const int64_t kspan = 1024;
    dim3 blk(32, 8);
    k_row_exponent<<<dim3((unsigned)ceil_div(m, 32), (unsigned)ceil_div(m, kspan)), blk, 0, s>>>(va, exb, kspan); count_launch();
    k_split<<<dim3((unsigned)(p.m_pad / 32), (unsigned)(p.k_pad / 32)), blk, 0, s>>>(va, exb, o.e, slices, p.m_pad,
                                                                                   p.k_pad, o.S, OZ_BM); count_launch();
    EVD_CUDA_TRY(cudaGetLastError());
  }
  *out = o;
  return EVD_OK;
}

size_t ozaki_presplit_gemm_bytes(int64_t m, int64_t n, int slices) {
  // B's slices and scales plus the split-K partials, for any offset (K <= m + OZ_BM)
  const int64_t kp = m + OZ_BM;
  const Pads p = pads(kp, n, kp);
  Carver c(nullptr);
  c.take<__nv_bfloat16>((size_t)slices * p.n_pad * p.k_pad);
  c.take<int>((size_t)p.n_pad);
  c.take<int>((size_t)p.n_pad);
  c.take<double>((size_t)splitk_count(kp, n, kp) * m * n);
  return c.off + 256;
}

evd_status_t ozaki_gemm_presplit(const Gemm& g, const SplitOperand& sa, int64_t off, void* scratch,
                                 size_t scratch_bytes, cudaStream_t s) {
  const int slices = sa.slices;
  if (g.ta != 'N' || g.lower || g.m != g.k || off < 0 || off % OZ_KS != 0 || off + g.m != sa.rows || g.n < 1)
    return EVD_ERR_INVALID_ARG;
  // the product starts on the row tile below `off`: its first e rows (and K-elements)
  // are computed against zero rows of B and not stored
  const int64_t off0 = off / OZ_BM * OZ_BM, e = off - off0;
  const int64_t mp = g.m + e, kp = g.k + e;
  const Pads p = pads(mp, g.n, kp);
  if (off0 + p.m_pad > sa.rows_pad || off0 + p.k_pad > sa.K_pad) return EVD_ERR_INVALID_ARG;
  Carver c(scratch);
  __nv_bfloat16* SB = c.take<__nv_bfloat16>((size_t)slices * p.n_pad * p.k_pad);
  int* exB = c.take<int>((size_t)p.n_pad);
  int* eB = c.take<int>((size_t)p.n_pad);
  const size_t base = c.off + 256;
  if (!scratch || scratch_bytes < base) return ws_fail(g.tag ? g.tag : "split product", scratch_bytes, base);
  int splits = splitk_count(mp, g.n, kp);
  while (splits > 1 && base + (size_t)splits * g.m * g.n * sizeof(double) > scratch_bytes) --splits;
  double* part = c.take<double>(splits > 1 ? (size_t)splits * g.m * g.n : 0);
  View vb;
  vb.p = g.B; vb.ld = g.ldb; vb.rows = g.n; vb.K = kp; vb.koff = e;
  vb.mode = (g.tb == 'N') ? 1 : 0;
  {
    StatScope sc(g.tag ? g.tag : "gemm", s, 0.0, 8.0 * (double)g.n * (double)g.k * 2.0 + 2.0 * slices * (double)p.n_pad * p.k_pad,
                 "tc_split_prep");
    dim3 blk(32, 8);
    if (p.k_pad <= 512) {
      const evd_status_t st = ensure_dynamic_smem((const void*)k_split_fused, 32 * (512 + 1) * sizeof(double));
      if (st != EVD_OK) return st;
      View va = vb;  // unused: every block takes B
      k_split_fused<<<dim3((unsigned)(p.n_pad / 32), 1u), 256, 32 * (p.k_pad + 1) * sizeof(double), s>>>(
          va, eB, SB, p.n_pad, vb, eB, SB, p.n_pad, 0, slices, p.k_pad); count_launch();
    } else {
      EVD_CUDA_TRY(cudaMemsetAsync(exB, 0, sizeof(int) * p.n_pad, s));
      const int64_t kspan = 1024;
      k_row_exponent<<<dim3((unsigned)ceil_div(g.n, 32), (unsigned)ceil_div(kp, kspan)), blk, 0, s>>>(vb, exB, kspan); count_launch();
      k_split<<<dim3((unsigned)(p.n_pad / 32), (unsigned)(p.k_pad / 32)), blk, 0, s>>>(vb, exB, eB, slices, p.n_pad,
                                                                                     p.k_pad, SB, OZ_BN); count_launch();
    }
    EVD_CUDA_TRY(cudaGetLastError());
  }
  MmaArgs a;
  a.SA = sa.S + (size_t)((off0 / OZ_BM) * (sa.K_pad / OZ_KS) + off0 / OZ_KS) * slices * (OZ_BM * OZ_KS);
  a.SB = SB;
  a.nkb = sa.K_pad / OZ_KS; a.nkb_b = p.k_pad / OZ_KS; a.c_skip = e;
  a.m = mp; a.n = g.n; a.s = slices; a.nst = (int)(p.k_pad / OZ_KS);
  uint32_t cols = 64;
  while (cols < (uint32_t)(slices * OZ_BN)) cols <<= 1;
  a.tmem_cols = cols;
  a.ea = sa.e + off0; a.eb = eB; a.C = g.C; a.ldc = g.ldc; a.alpha = g.alpha; a.beta = g.beta;
  a.lower = 0; a.batched = 0; a.bm_pad = p.m_pad; a.bn_pad = p.n_pad; a.sC = 0; a.m_first = -1;
  a.stages_per_split = (int)ceil_div(ceil_div(a.nst, splits), OZ_PERIOD) * OZ_PERIOD;
  const int zsplits = (int)ceil_div(a.nst, a.stages_per_split);
  a.part = (zsplits > 1) ? part : nullptr;
  a.st = g.status ? g.status : standalone_status();
  if (!a.st) return EVD_ERR_OOM;
  {
    const evd_status_t st = ensure_dynamic_smem(mma_kernel(slices), smem_bytes(OZ_MAXS));
    if (st != EVD_OK) return st;
  }
  dim3 grid((unsigned)(p.m_pad / OZ_BM), (unsigned)(p.n_pad / OZ_BN), (unsigned)zsplits);
  if (grid.y > 65535) return EVD_ERR_INVALID_ARG;
  StatScope sc(g.tag ? g.tag : "gemm", s, 2.0 * (double)mp * g.n * kp * (double)(slices * (slices + 1) / 2), 0.0,
               "tc_split");
  void* kargs[] = {&a};
  EVD_CUDA_TRY(cudaLaunchKernel(mma_kernel(slices), grid, dim3(OZ_THREADS), kargs, smem_bytes(slices), s)); count_launch();
  EVD_CUDA_TRY(cudaGetLastError());
  if (zsplits > 1) {
    for (int64_t j0 = 0; j0 < g.n; j0 += 65535) {
      const int64_t cols2 = std::min<int64_t>(g.n - j0, 65535);
      k_splitk_reduce<<<dim3((unsigned)std::min<int64_t>(ceil_div(g.m, 256), 16), (unsigned)cols2), 256, 0, s>>>(
          part + j0 * g.m, zsplits, g.m, g.n, g.alpha, g.beta, g.C + j0 * g.ldc, g.ldc, 0); count_launch();
    }
    EVD_CUDA_TRY(cudaGetLastError());
  }
  return EVD_OK;
}

}  // namespace evd
