// BC back-transformation, one wave per launch, fused (Sec. 2.1.2, blocked form).
//
// For the groups G_p of one wave (row-disjoint, see evd_back.cu) and X = Q:
//     W_p^T = X_p^T V_p          (n x g, K = h rows of the group)
//     X_p  -= Y_p W_p            (Y_p = V_p T_p)
// with X_p = X(R0_p : R0_p + h, :), R0_p = R0_0 - p (g + b).  One CTA owns group p
// and 128 columns c0 .. c0+127 of X and does both products on the tensor cores
// as split products with exact integer accumulation:
//   phase 1  D1[m][i] = sum_r X(R0+r, c0+m) V(r, i)          M = 128, N = g = 64, K = 128
//            The CTA's converter warps read the fixed-point tile of X, write its
//            digits straight into shared memory; V's slices come pre-split.
//   exact    D1 drained into exact 128-bit integer sums (W^T times a power of two).
//   phase 2  D2[r][c] = sum_i Y(r, i) W(i, c)                 M = 128 rows, N = 128
//            columns (two halves of 64), K = g = 64.  W is split in the CTA straight
//            from the integer sums (scale per column of X, integer rescaling and
//            rounding), Y's slices come pre-split; X(R0 + r, c0 + c) -= D2[r][c].
//            The accumulator's lanes are rows of X, so each warp of the epilogue
//            reads and writes 32 consecutive elements of one column.
// Digits: S balanced base-256 digits per operand held as float16 (exact for
// integers up to 2048).  Both products have K <= 128, so every FP32 accumulator
// of the slice pairs t + u = k stays an exact integer below 2^24 (at most
// (k + 1) 128 128^2 with digits in [-128, 128]).  S = 7 digits carry 55 bits
// (the 8 bfloat16 slices of 7 bits of the general product, evd_ozaki.cu, carry 56)
// with 28 slice-pair products in place of 36; a digit is a byte of the offset
// integer, taken with one byte permute.
// X is kept in fixed point during BC-Back: T = round(x 2^(8S - 1)) in int64, in
// place of the FP64 values (bcback_fixed_point converts on entry and exit).  X is
// orthogonal (D&C's eigenvectors times orthogonal reflectors), so |x| <= 1 and
// |T| <= 2^(8S - 1).  The split of the X operand is then the integer itself and
// each update is an exact 128-bit rescale and one int64 subtraction; every update
// rounds once to the grid 2^(1-8S) (2^-55 at S = 7, far below FP64's product
// error over the 2n/b waves).  Only the int64 tile of X moves through HBM (read
// twice, written once): no slice or W buffer is materialized in global memory.
//
// Roles (576 threads): warp 0 copies (tensor copies of X, up to five K-steps
// ahead, and the pre-split blobs), warp 1 owns the tensor memory (512 columns) and
// issues the MMAs, warps 2..17 convert X and W into digits and drain the
// accumulators (16 accumulator columns per thread).  Every wait is bounded.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "device_util.cuh"
#include "evd_internal.h"
#include "evd_ozaki.h"
#include "tc_common.cuh"

namespace evd {

namespace {

using namespace tcx;

constexpr int BB_G = 64;          // group size g = b
constexpr int BB_H = 128;         // padded rows of a group (h = 2b - 1 = 127)
constexpr int BB_THREADS = 576;  // warp 0 copies, warp 1 MMA, warps 2..17 convert and drain
constexpr int BB_P1_STAGES = 3;
constexpr int BB_XROWS = OZ_KS + 2;                       // rows of an X box (starts on an even row)
constexpr uint32_t BB_XS = BB_XROWS * OZ_BM * 8;          // one X K-step in shared memory (int64)

__device__ __forceinline__ int biased_exp(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}
__device__ __forceinline__ int frexp_exp(int biased_max) { return (biased_max > 0) ? biased_max - 1022 : -1022; }

// ---------------------------------------------------------------- 8-bit digits
// An operand x with frexp exponent e (|x| < 2^e) is the integer
// T = round_half_away(x 2^(8S - 1 - e)), |T| <= 2^(8S - 1).  With the offset
// O = 128 (1 + 256 + ... + 256^(S-2)), digit j < S - 1 (from the bottom) of T is
// byte j of T + O minus 128, in [-128, 127]; the top digit is (T + O) >> 8(S - 1),
// in [-128, 128].  Slice t holds digit S - 1 - t (slice 0 is the top).
template <int S>
__host__ __device__ constexpr long long offset8() {
  long long o = 0;
  for (int j = 0; j < S - 1; ++j) o = (o << 8) + 128;
  return o;
}

// round_half_away(x 2^p) as an integer (|x 2^p| < 2^62): the general product's
// scaling with no slices, T = x 2^(0 - e) for e = -p.
__device__ __forceinline__ long long scaled_pow2(double x, int p) { return ozaki_scaled(x, -p, 0); }

__device__ __forceinline__ uint32_t hsub2_bits(uint32_t a, uint32_t b) {
  const __half2 v = __hsub2(*reinterpret_cast<const __half2*>(&a), *reinterpret_cast<const __half2*>(&b));
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Digit j (0..3 within its 32-bit word) of two offset integers as a float16 pair:
// the byte f placed under the float16 exponent of 1024 (bits 0x6400 | f, the value
// 1024 + f exactly), minus 1152 gives the digit f - 128 exactly.
__device__ __forceinline__ uint32_t digit8_pair(uint32_t wa, uint32_t wb, int j) {
  const uint32_t f = __byte_perm(wa, wb, (uint32_t)j | ((uint32_t)(4 + j) << 8));
  return hsub2_bits((f & 0x00FF00FFu) | 0x64006400u, 0x64806480u);
}

// The top digits d in [-128, 128] of two offset integers as a float16 pair: the
// bits 0x6480 + d are the float16 1152 + d, minus 1152 gives d.
__device__ __forceinline__ uint32_t top8_pair(long long TOa, long long TOb, int sh) {
  const uint32_t a = (uint32_t)(0x6480 + (int)(TOa >> sh)), b = (uint32_t)(0x6480 + (int)(TOb >> sh));
  return hsub2_bits(__byte_perm(a, b, 0x5410), 0x64806480u);
}

// Slice tt of NV offset integers TO (NV even) as NV / 2 float16 pairs.
template <int S, int NV>
__device__ __forceinline__ void slice8(const long long* TO, int tt, uint32_t* w) {
#pragma unroll
  for (int q = 0; q < NV / 2; ++q) {
    if (tt == 0) {
      w[q] = top8_pair(TO[2 * q], TO[2 * q + 1], 8 * (S - 1));
    } else {
      const int j = S - 1 - tt;  // digit position from the bottom
      const uint32_t wa = (j < 4) ? (uint32_t)TO[2 * q] : (uint32_t)((unsigned long long)TO[2 * q] >> 32);
      const uint32_t wb = (j < 4) ? (uint32_t)TO[2 * q + 1] : (uint32_t)((unsigned long long)TO[2 * q + 1] >> 32);
      w[q] = digit8_pair(wa, wb, j & 3);
    }
  }
}

// ---------------------------------------------------------------- prep
// The compact WY factors of the wave's groups, with the dense products on the
// tensor cores:
//   k_bb_gather   V_p (128 x g, zero outside the parallelogram, rows >= h zero), tau_p
//   product       G_p = V_p^T V_p                         (batched split product)
//   k_bb_T        T_p upper triangular with H_0 ... H_{g-1} = I - V T V^T:
//                 T(i, i) = tau_i, T(0:i, i) = -tau_i T(0:i, 0:i) G(0:i, i)
//   product       Y_p = V_p T_p                           (batched split product)
//   k_bb_split    8-bit float16 slices of V (B operand of phase 1: N = i, K = r,
//                 scale per i) and of Y (A operand of phase 2: M = r, K = i, scale
//                 per r)
// Problem p of wave t is the group J' = jp0 + p, J = nJ - 1 - J', k = t - J'.
__global__ void __launch_bounds__(256) k_bb_gather(const double* __restrict__ U, const double* __restrict__ Utau,
                                                   int64_t n, int b, const int2* __restrict__ gjk, double* Vg,
                                                   double* taug) {
  constexpr int g = BB_G, H = BB_H;
  const int64_t pidx = blockIdx.x;
  const int64_t J = gjk[pidx].x, k = gjk[pidx].y;
  double* V = Vg + (size_t)pidx * H * g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < g; i += 8) {
    const int64_t j = J * g + i;
    int64_t idx = -1;
    int m = 0;
    if (j < n - 2 && k < (n - 3 - j) / b + 1) {
      // sweep_offset(n, b, j) + k with F(T) = sum_{s=0}^{T} floor(s / b)
      auto F = [&](int64_t T0) -> int64_t {
        if (T0 < 0) return 0;
        const int64_t q = T0 / b;
        return (int64_t)b * q * (q - 1) / 2 + q * (T0 - q * b + 1);
      };
      idx = F(n - 3) - F(n - 3 - j) + j + k;
      const int64_t r0 = j + 1 + k * b;
      m = (int)((r0 + b - 1 < n - 1) ? b : n - r0);
    }
    for (int r = lane; r < H; r += 32) {
      const int q = r - i;  // reflector i occupies rows i .. i + m - 1
      V[r + (size_t)i * H] = (idx >= 0 && q >= 0 && q < m) ? U[idx * b + q] : 0.0;
    }
    if (lane == 0) taug[pidx * g + i] = (idx >= 0) ? Utau[idx] : 0.0;
  }
}

__global__ void __launch_bounds__(64) k_bb_T(const double* __restrict__ Gg, const double* __restrict__ taug,
                                             double* Tg) {
  constexpr int g = BB_G;
  extern __shared__ double tsm[];
  double* G = tsm;          // g x g
  double* T = tsm + g * g;  // g x g
  const int q = threadIdx.x;
  const int64_t pidx = blockIdx.x;
  for (int idx = q; idx < g * g; idx += g) {
    G[idx] = Gg[(size_t)pidx * g * g + idx];
    T[idx] = 0.0;
  }
  __syncthreads();
  for (int i = 0; i < g; ++i) {
    const double ti = taug[pidx * g + i];
    double s = 0.0;
    if (q < i)
      for (int l = q; l < i; ++l) s += T[q + l * g] * G[l + i * g];
    __syncthreads();
    if (q < i) T[q + i * g] = -ti * s;
    if (q == i) T[q + i * g] = ti;
    __syncthreads();
  }
  for (int idx = q; idx < g * g; idx += g) Tg[(size_t)pidx * g * g + idx] = T[idx];
}

template <int S>
__global__ void __launch_bounds__(256) k_bb_split(const double* __restrict__ Vg, const double* __restrict__ Yg,
                                                  __half* Vb, int* eV, __half* Yb, int* eY) {
  constexpr int g = BB_G, H = BB_H;
  constexpr long long off = offset8<S>();
  __shared__ int ex_s[H];
  const int tid = threadIdx.x;
  const int64_t pidx = blockIdx.x;
  const double* V = Vg + (size_t)pidx * H * g;
  const double* Y = Yg + (size_t)pidx * H * g;
  if (tid < g) {
    int mx = 0;
    for (int r = 0; r < H; ++r) mx = max(mx, biased_exp(V[r + (size_t)tid * H]));
    eV[pidx * g + tid] = frexp_exp(mx);
    ex_s[tid] = frexp_exp(mx);
  }
  __syncthreads();
  __half* Vp = Vb + (size_t)pidx * S * g * H;
  for (int u = tid; u < g * H / 8; u += 256) {
    const int i = u / (H / 8), r0 = (u % (H / 8)) * 8;
    long long TO[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) TO[q] = scaled_pow2(V[(r0 + q) + (size_t)i * H], 8 * S - 1 - ex_s[i]) + off;
#pragma unroll
    for (int tt = 0; tt < S; ++tt) {
      uint32_t w[4];
      slice8<S, 8>(TO, tt, w);
      *reinterpret_cast<uint4*>(Vp + blob_index(i, r0, tt, S, 64, H / 16)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  __syncthreads();
  if (tid < H) {
    int mx = 0;
    for (int i = 0; i < g; ++i) mx = max(mx, biased_exp(Y[tid + (size_t)i * H]));
    eY[pidx * H + tid] = frexp_exp(mx);
    ex_s[tid] = frexp_exp(mx);
  }
  __syncthreads();
  __half* Yp = Yb + (size_t)pidx * S * H * g;
  for (int u = tid; u < H * g / 8; u += 256) {
    const int r = u / (g / 8), i0 = (u % (g / 8)) * 8;
    long long TO[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) TO[q] = scaled_pow2(Y[r + (size_t)(i0 + q) * H], 8 * S - 1 - ex_s[r]) + off;
#pragma unroll
    for (int tt = 0; tt < S; ++tt) {
      uint32_t w[4];
      slice8<S, 8>(TO, tt, w);
      *reinterpret_cast<uint4*>(Yp + blob_index(r, i0, tt, S, 128, g / 16)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// ---------------------------------------------------------------- fused wave
constexpr int BB_NX = 5;    // X boxes in flight: the tensor copies of X run up to five K-steps ahead
constexpr int BB_MAXS = 7;  // digits of the waves (both precisions)

struct WaveArgs {
  CUtensorMap xmap;  // X as a 2-D int64 tensor (rows, columns), box BB_XROWS x 128
  long long* X;     // X in fixed point: x = T 2^(1 - 8S) (see bcback_fixed_point)
  int64_t ldx, n;
  int64_t R0;       // first row of group 0
  int64_t gstride;  // rows between consecutive groups (g + b)
  int h0;           // rows of group 0 (the others have h)
  int h;            // rows of a group (2b - 1)
  const __half* Vb;
  const int* eV;
  const __half* Yb;
  const int* eY;
  int* st;
  int64_t tile0;       // column tile of blockIdx.x = 0 (tiles of 128 columns)
  const int2* ranges;  // per group: the column tiles [x, y] that can be nonzero in its rows (nullptr: all)
};

// AND of a predicate over the 512 threads of warps 2..17 (named barrier 1).
__device__ __forceinline__ bool bar_and_epi(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, 512, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)(v ? 1 : 0))
      : "memory");
  return r != 0;
}

// The exact signed 128-bit value (hi, lo) of one accumulator pair:
// R = Rh 2^(8 (L - H)) + Rl.
template <int S>
__device__ __forceinline__ void sum128(long long rh, long long rl, long long& hi, unsigned long long& lo) {
  constexpr int L = S - 1, H = (L < 3) ? L : 3, shift_hi = 8 * (L - H);
  lo = (shift_hi == 0) ? (unsigned long long)rh : ((unsigned long long)rh << shift_hi);
  hi = (shift_hi == 0) ? (rh >> 63) : (rh >> (64 - shift_hi));
  if (L >= 4) {
    const unsigned long long nlo = lo + (unsigned long long)rl;
    hi += (rl >> 63) + (nlo < lo ? 1 : 0);
    lo = nlo;
  }
}

// 64-bit shifts with PTX semantics: an amount above 64 (a negative int passed as
// unsigned included) is clamped to 64, which gives 0.
__device__ __forceinline__ unsigned long long shl64(unsigned long long x, uint32_t k) {
  unsigned long long r;
  asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(k));
  return r;
}
__device__ __forceinline__ unsigned long long shr64(unsigned long long x, uint32_t k) {
  unsigned long long r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(k));
  return r;
}

// 64-bit arithmetic shift right with PTX semantics: an amount above 64 is clamped to
// 64, which gives the sign fill.
__device__ __forceinline__ long long sar64(long long x, uint32_t k) {
  long long r;
  asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(k));
  return r;
}

// T = floor(R 2^d + 1/2), R = hi 2^64 + lo signed 128-bit, |R 2^d| < 2^62: round to
// nearest, ties toward +infinity.  d >= 0: R sits in the low word, shift it left.
// d = -k < 0: add 2^(k-1) in two's complement and shift right arithmetically by k;
// k >= 127 gives 0 (|R| < 2^126).  Branch-free: shift amounts out of range clamp.
__device__ __forceinline__ long long round_shift(long long hi, unsigned long long lo, int d) {
  const uint32_t k = (uint32_t)(-d);
  const unsigned long long nl = lo + shl64(1ull, k - 1u);
  const long long nh = hi + (long long)shl64(1ull, k - 65u) + (nl < lo ? 1ll : 0ll);
  const long long low = (long long)(shr64(nl, k) | shl64((unsigned long long)nh, 64u - k));
  const long long high = sar64(nh, k - 64u);
  const long long r = (k >= 127u) ? 0ll : ((k < 64u) ? low : high);
  return (d >= 0) ? (long long)shl64(lo, (uint32_t)d) : r;
}

// R = Rh 2^G + Rl (G = 8 (L - H)) without forming the 128-bit value:
// floor(R 2^-k + 1/2) for 0 < k < G, where Rh 2^G is a multiple of 2^k and only the
// low part rounds (|result| < 2^62).
template <int G>
__device__ __forceinline__ long long round_split(long long Rh, long long Rl, int k) {
  return (long long)((unsigned long long)Rh << (G - k)) + ((Rl + (1ll << (k - 1))) >> k);
}
// The bit length of the one's complement of R = Rh 2^G + Rl: that of |R| for R >= 0
// and of |R| - 1 for R < 0 (one less than |R|'s only when |R| is a power of two); 0
// for R = 0 and R = -1.  With s = floor(R / 2^G) = Rh + (Rl >> G) it is s's plus G
// unless s is 0 or -1, when R itself fits in G + 1 bits.
__device__ __forceinline__ int bitlen64(long long x) { return 64 - __clzll(x ^ (x >> 63)); }
template <int G>
__device__ __forceinline__ int bitlen_split(long long Rh, long long Rl) {
  const long long s = Rh + (Rl >> G);
  const long long r = (long long)((unsigned long long)s << G) + (Rl & ((1ll << G) - 1));
  return (s != 0 && s != -1) ? bitlen64(s) + G : bitlen64(r);
}

// The exact integer value of an FP32 accumulator v with |v| < 2^22: v + 1.5 * 2^23
// lies in [2^23, 2^24), where the float's ulp is 1, so the integer is its low
// mantissa bits: bits(v + 1.5 * 2^23) - 0x4B400000.
constexpr uint32_t kMagicBits = 0x4B400000u;

// d = a * b + c with a 32 x 32 -> 64-bit multiply (the FMA pipe's wide multiply-add),
// modulo 2^64.
__device__ __forceinline__ unsigned long long mad_wide_u32(uint32_t a, uint32_t b, unsigned long long c) {
  unsigned long long d;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

// Weight 2^(8 (H - k)) of diagonal k in Rh (k <= H) or 2^(8 (L - k)) in Rl.
template <int S>
__host__ __device__ constexpr uint32_t weight8(int k) {
  return 1u << (k <= ((S - 1 < 3) ? S - 1 : 3) ? 8 * (((S - 1 < 3) ? S - 1 : 3) - k) : 8 * (S - 1 - k));
}
// The starting value of Rh (high) or Rl that cancels the magic offset of the add
// trick: -0x4B400000 times the sum of the weights.
template <int S>
__host__ __device__ constexpr long long magic_start8(bool high) {
  long long w = 0;
  for (int k = 0; k < S; ++k)
    if ((k <= ((S - 1 < 3) ? S - 1 : 3)) == high) w += weight8<S>(k);
  return -(long long)kMagicBits * w;
}

// Drain the S weight accumulators of this thread's 16 columns (TMEM lane quadrant
// `quad`, columns 16 q4 .. +15 of each weight) into the two exact sums
//   Rh = sum_{k <= H} acc_k 2^(8 (H - k)),   Rl = sum_{k > H} acc_k 2^(8 (L - k)),
// every value by the add trick: its float's bits weighted by a wide multiply-add,
// the starting values cancelling the magic offset.  The trick is exact while
// v + 1.5 * 2^23 stays in [2^23, 2^24) (|v| <= 2^22), but an accumulator may reach
// (k + 1) K 2^14, up to 2^24 (K <= KMAX): for the diagonals whose bound reaches
// 2^22, where a sum left that binade (its exponent field changed) for any lane of the
// warp, the warp reads the 16 values again and replaces the trick's term by the
// hardware conversion, exact below 2^24.
template <int S, int KMAX>
__device__ __forceinline__ void drain16(uint32_t tmem, int quad, int q4, long long* Rh, long long* Rl) {
  constexpr int L = S - 1, H = (L < 3) ? L : 3;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    Rh[c] = magic_start8<S>(true);
    Rl[c] = magic_start8<S>(false);
  }
#pragma unroll
  for (int k = 0; k <= L; ++k) {
    const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(k * OZ_BN + q4 * 16);
    float v[16];
    tc_ld16(taddr, v);
    const uint32_t wk = weight8<S>(k);
    uint32_t bad = 0;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const uint32_t bv = __float_as_uint(v[c] + 12582912.0f);
      if ((long long)(k + 1) * KMAX * 16384 >= (1ll << 22)) bad |= bv ^ 0x4B000000u;  // else below 2^22 by the bound
      long long& acc = (k <= H) ? Rh[c] : Rl[c];
      acc = (long long)mad_wide_u32(bv, wk, (unsigned long long)acc);
    }
    if (__any_sync(0xffffffffu, (bad >> 23) != 0)) {
      tc_ld16(taddr, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        long long& acc = (k <= H) ? Rh[c] : Rl[c];
        acc += (long long)wk * ((long long)__float2int_rn(v[c]) -
                                ((long long)__float_as_uint(v[c] + 12582912.0f) - (long long)kMagicBits));
      }
    }
  }
}

// Write the S digit slices of NV consecutive K-values (already scaled integers T,
// NV = 4 or 8, kk0 a multiple of NV) into a K-major blob of TR-row tiles: row m,
// K-elements kk0 .. kk0+NV-1 of the blob's K-step.
template <int S, int NV, int TR>
__device__ __forceinline__ void put_digits(uint8_t* blob_ks, int m, int kk0, const long long* T) {
  constexpr long long off = offset8<S>();
  const int core = ((m >> 3) * 2 + (kk0 >> 3)) * 64 + (m & 7) * 8 + (kk0 & 7);  // elements
  long long TO[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) TO[q] = T[q] + off;
#pragma unroll
  for (int tt = 0; tt < S; ++tt) {
    uint32_t w[NV / 2];
    slice8<S, NV>(TO, tt, w);
    uint8_t* dst = blob_ks + ((size_t)tt * TR * OZ_KS + core) * 2;
    if (NV == 8) *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2 % (NV / 2)], w[3 % (NV / 2)]);
    else *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
  }
}

// 576 threads are 18 warps, so some of the SM's four sub-partitions hold 5 warps and
// their 16K registers allow at most 96 per thread.
template <int S>
__global__ void __launch_bounds__(BB_THREADS, 1) k_bcback_wave(const __grid_constant__ WaveArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr uint32_t A_KS = S * OZ_BM * OZ_KS * 2;   // one K-step of a 128-row operand (all slices)
  constexpr uint32_t B_KS = S * OZ_BN * OZ_KS * 2;   // one K-step of a 64-row operand
  constexpr int NK = BB_H / OZ_KS;                    // K-steps of phase 1
  constexpr int G = 8 * ((S - 1) - ((S - 1 < 3) ? S - 1 : 3));  // R = Rh 2^G + Rl
  // phase 1: A stages [0, 3 A_KS), B stages, then the BB_NX X boxes; phase 2: Y (all
  // K-steps) at 0, one half of W (64 columns, all K-steps) after it
  constexpr uint32_t P1_B = BB_P1_STAGES * A_KS;
  constexpr uint32_t P1_X = P1_B + BB_P1_STAGES * B_KS;
  constexpr uint32_t P2_Y = 0;
  constexpr uint32_t P2_W = 4 * A_KS;
  constexpr uint32_t DATA = (P1_X + BB_NX * BB_XS > P2_W + 4 * B_KS) ? P1_X + BB_NX * BB_XS : P2_W + 4 * B_KS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + DATA);
  uint64_t* fullA = bars;                          // [3], 16 arrivals (converter warps)
  uint64_t* fullB = bars + 3;                      // [3], 1 arrival + bytes
  uint64_t* empty = bars + 6;                      // [3], MMA commit
  uint64_t* acc1 = bars + 9;                       // phase 1 accumulators ready
  uint64_t* fullW = bars + 10;                     // W half written (8 arrivals), two phases
  uint64_t* fullY = bars + 11;                     // Y copied (1 arrival + bytes)
  uint64_t* acc2 = bars + 12;                      // phase 2 half ready (two phases)
  uint64_t* drained = bars + 13;                   // epilogue drained phase 2 half 0 (16 arrivals)
  uint64_t* fullX = bars + 14;                     // [BB_NX], X box landed (1 arrival + bytes)
  uint64_t* xfree = fullX + BB_NX;                 // [BB_NX], X box read by the converters (16 arrivals)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(xfree + BB_NX);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* eVs = reinterpret_cast<int*>(tmem_slot + 4);        // 64
  int* eYs = eVs + BB_G;                                     // 128
  int* exw = eYs + BB_H;                                     // 4 x 128 (per-quarter maxima)
  int* eWs = exw + 4 * BB_H;                                 // 128, scale of W per column of X
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = blockIdx.y;
  const int64_t tile = a.tile0 + blockIdx.x;
  if (a.ranges) {
    // X's rows of this group are zero in this column tile (BC-Back of the identity):
    // W and the update vanish.  The whole CTA leaves before any set-up.
    const int2 r = a.ranges[p];
    if (tile < r.x || tile > r.y) return;
  }
  const int64_t c0 = tile * OZ_BM;
  const int64_t R0 = a.R0 - p * a.gstride;
  const int hp = (p == 0) ? a.h0 : a.h;
  const __half* Vp = a.Vb + (size_t)p * S * BB_G * BB_H;
  const __half* Yp = a.Yb + (size_t)p * S * BB_H * BB_G;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 3; ++i) {
      mbar_init(smem_u32(fullA + i), 16);
      mbar_init(smem_u32(fullB + i), 1);
      mbar_init(smem_u32(empty + i), 1);
    }
    for (int i = 0; i < BB_NX; ++i) {
      mbar_init(smem_u32(fullX + i), 1);
      mbar_init(smem_u32(xfree + i), 16);
    }
    mbar_init(smem_u32(acc1), 1);
    mbar_init(smem_u32(fullW), 8);
    mbar_init(smem_u32(fullY), 1);
    mbar_init(smem_u32(acc2), 1);
    mbar_init(smem_u32(drained), 16);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < BB_G) eVs[threadIdx.x] = a.eV[p * BB_G + threadIdx.x];
  if (threadIdx.x < BB_H) eYs[threadIdx.x] = a.eY[p * BB_H + threadIdx.x];
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- copies: the X box of K-step jx (tensor copy: rows x0 .. x0 + 17
      // from the even row x0 = R0 + 16 jx - (R0 & 1), columns c0 .. c0 + 127, zero
      // outside X) once the converters have read the box BB_NX K-steps back, and V's
      // slices of K-step jv once the MMAs are done with its stage.  X goes first: its
      // copies run BB_NX K-steps ahead of the converters, V's three.
      const uint64_t xmap = reinterpret_cast<uint64_t>(&a.xmap);
      int jx = 0, jv = 0;
      long long spins = 0;
      while ((jx < NK || jv < NK) && !*abort) {
        if (jx < NK && (jx < BB_NX || mbar_try(smem_u32(xfree + jx % BB_NX), ((jx / BB_NX) - 1) & 1))) {
          const int xi = jx % BB_NX;
          mbar_expect_tx(smem_u32(fullX + xi), BB_XS);
          const int x0 = (int)(R0 + (int64_t)jx * OZ_KS - (R0 & 1)), y0 = (int)c0;
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
              ::"r"(smem_u32(smem + P1_X + xi * BB_XS)), "l"(xmap), "r"(x0), "r"(y0), "r"(smem_u32(fullX + xi))
              : "memory");
          ++jx;
          continue;
        }
        if (jv < NK && (jv < 3 || mbar_try(smem_u32(empty + jv % 3), ((jv / 3) - 1) & 1))) {
          const int si = jv % 3;
          mbar_expect_tx(smem_u32(fullB + si), B_KS);
          bulk_load(smem_u32(smem + P1_B + si * B_KS), Vp + (size_t)jv * S * OZ_BN * OZ_KS, B_KS,
                    smem_u32(fullB + si));
          ++jv;
          continue;
        }
        if (++spins > OZ_WAIT_LIMIT) {
          *abort = 1;
          dev_set_status(a.st, EVD_ERR_TIMEOUT, 9100);
        }
      }
      if (*abort) {
        // let the copies already in flight land before the CTA exits
        for (int j = (jx > BB_NX ? jx - BB_NX : 0); j < jx; ++j)
          for (long long i = 0; i < OZ_WAIT_LIMIT && !mbar_try(smem_u32(fullX + j % BB_NX), (j / BB_NX) & 1); ++i) {}
        for (int j = (jv > 3 ? jv - 3 : 0); j < jv; ++j)
          for (long long i = 0; i < OZ_WAIT_LIMIT && !mbar_try(smem_u32(fullB + j % 3), (j / 3) & 1); ++i) {}
      }
      // phase 1 finished reading shared memory before the Y copy may overwrite it
      if (!*abort && mbar_wait(smem_u32(acc1), 0, abort, a.st, 9102)) {
        mbar_expect_tx(smem_u32(fullY), 4 * A_KS);
        bulk_load(smem_u32(smem + P2_Y), Yp, 4 * A_KS, smem_u32(fullY));
        mbar_wait(smem_u32(fullY), 0, abort, a.st, 9104);  // let the copy land before leaving
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issue
      const uint64_t dbase = desc_kmajor(smem_u32(smem));
      bool ok = true;
      for (int j = 0; j < NK && ok; ++j) {
        const int si = j % 3, round = j / 3;
        ok = mbar_wait(smem_u32(fullA + si), round & 1, abort, a.st, 9111) &&
             mbar_wait(smem_u32(fullB + si), round & 1, abort, a.st, 9112);
        if (!ok) break;
        tc_fence_after();
        issue_stage<S, true>(tmem, dbase + (uint64_t)((si * A_KS) >> 4),
                             dbase + (uint64_t)((P1_B + si * B_KS) >> 4), j > 0 ? 1u : 0u);
        tc_commit(smem_u32(empty + si));
      }
      if (ok) tc_commit(smem_u32(acc1));
      // phase 2, half 0 then half 1 (the epilogue drains half 0 in between)
      for (int hf = 0; hf < 2 && ok; ++hf) {
        if (hf == 0) ok = mbar_wait(smem_u32(fullY), 0, abort, a.st, 9113);
        if (ok) ok = mbar_wait(smem_u32(fullW), hf, abort, a.st, 9114);
        if (ok && hf == 1) ok = mbar_wait(smem_u32(drained), 0, abort, a.st, 9115);
        if (!ok) break;
        tc_fence_after();
        for (int ks = 0; ks < BB_G / OZ_KS; ++ks)
          issue_stage<S, true>(tmem, dbase + (uint64_t)((P2_Y + ks * A_KS) >> 4),
                               dbase + (uint64_t)((P2_W + ks * B_KS) >> 4), ks > 0 ? 1u : 0u);
        tc_commit(smem_u32(acc2));
      }
    }
  } else {
    // ---------------- converter / epilogue warps 2..17 (512 threads)
    // Every thread of these warps passes through the same named barriers whatever
    // happens (a bounded wait that gives up only clears `ok`), and `ok` is made
    // uniform at each of them, so no thread can be left waiting at a barrier.
    const int ct = threadIdx.x - 64;
    // phase 1 producer mapping: column m = ct / 4, rows 4 kq .. 4 kq + 3 of a K-step
    const int m = ct >> 2, kq = ct & 3;
    // X is held in fixed point on the grid 2^(1 - 8S): the split of the X operand
    // (frexp exponent 0, |x| <= 1) is then the integer itself.
    const int xoff = (int)(R0 & 1);  // row R0 + 16 j sits at row xoff of its box
    bool ok = true;
    for (int j = 0; j < NK; ++j) {
      const int si = j % 3, round = j / 3, xi = j % BB_NX;
      long long T[4];
      if (ok) ok = mbar_wait(smem_u32(fullX + xi), (j / BB_NX) & 1, abort, a.st, 9120);
      const long long* xs = reinterpret_cast<const long long*>(smem + P1_X + xi * BB_XS) + m * BB_XROWS + kq * 4 + xoff;
#pragma unroll
      for (int q = 0; q < 4; ++q) T[q] = (ok && j * OZ_KS + kq * 4 + q < hp) ? xs[q] : 0ll;
      // the reads of the box (generic proxy) are ordered before the tensor copy that
      // refills it (async proxy) by a proxy fence in every reading thread
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(xfree + xi));  // the box may be refilled
      if (ok && round > 0) ok = mbar_wait(smem_u32(empty + si), (round - 1) & 1, abort, a.st, 9121);
      if (ok) put_digits<S, 4, OZ_BM>(smem + si * A_KS, m, kq * 4, T);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      ok = __all_sync(0xffffffffu, ok);
      if (ok && lane == 0) mbar_arrive(smem_u32(fullA + si));
    }
    // phase 1 result: W^T(m2, i), i = 16 q4 .. +15, as exact 128-bit integers R with
    // W^T = R 2^(eV_i - 8S - 6) (X on the grid 2^(1 - 8S), V_i's digits scaled by
    // 2^(8S - 1 - eV_i), the diagonal sums weighted from the lowest diagonal up)
    const int quad = warp & 3, q4 = (warp - 2) >> 2;
    const int m2 = quad * 32 + lane;
    if (ok) ok = mbar_wait(smem_u32(acc1), 0, abort, a.st, 9122);
    ok = bar_and_epi(ok);
    long long Rh[16], Rl[16];
    int eW = -1022;
    {
      int bmax = -100000;  // max over this thread's columns of bitlen(R) + scale
      if (ok) {
        tc_fence_after();
        drain16<S, BB_H - 1>(tmem, quad, q4, Rh, Rl);
        tc_fence_before();
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          // one's complement bit length: a negative power of two scales to exactly
          // -2^(8S - 1), a top digit of -128, which the digits allow
          const int bl = bitlen_split<G>(Rh[c], Rl[c]);
          if (bl > 0) bmax = max(bmax, bl + eVs[q4 * 16 + c] - 8 * S - 6);
        }
      }
      // row scale of W^T over its 64 columns (the four quarters meet in shared memory)
      exw[q4 * BB_H + m2] = bmax;
      ok = bar_and_epi(ok);
      const int e4 = max(max(exw[m2], exw[BB_H + m2]), max(exw[2 * BB_H + m2], exw[3 * BB_H + m2]));
      eW = (e4 > -100000) ? e4 : -1022;
    }
    if (q4 == 0) eWs[m2] = eW;
    // W(i, m2), i = 16 q4 .. +15, as the integers round(W 2^(8S - 1 - eW)) of its
    // column's scale (integer rescaling of the exact sums, no FP64 round trip):
    // K-step q4 of the B operand of phase 2, half m2 / 64 of the columns
    long long T[16];
    if (ok) {
      // T = round(R 2^-k), k = eW + 7 - eV_i: by the split form when every lane's k
      // lies in (0, G) or its R is zero (a zero column of V, or a zero row of W^T:
      // the scale marker -1022), else through the 128-bit value
      bool fast = true;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int k = eW + 7 - eVs[q4 * 16 + c];
        const bool zero = eW == -1022 || eVs[q4 * 16 + c] == -1022;
        fast &= zero | ((k > 0) & (k < G));
      }
      if (__all_sync(0xffffffffu, fast)) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const bool zero = eW == -1022 || eVs[q4 * 16 + c] == -1022;
          const long long t = round_split<G>(Rh[c], Rl[c], zero ? 1 : eW + 7 - eVs[q4 * 16 + c]);
          T[c] = zero ? 0ll : t;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          long long hi;
          unsigned long long lo;
          sum128<S>(Rh[c], Rl[c], hi, lo);
          T[c] = round_shift(hi, lo, eVs[q4 * 16 + c] - 7 - eW);
        }
      }
    }
    const bool upper = quad >= 2;  // columns 64 .. 127: written once half 0's products are done
    if (ok && !upper) {
      put_digits<S, 8, OZ_BN>(smem + P2_W + q4 * B_KS, m2, 0, T);
      put_digits<S, 8, OZ_BN>(smem + P2_W + q4 * B_KS, m2, 8, T + 8);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(fullW));
    }
    ok = bar_and_epi(ok);  // eWs complete
    // phase 2: X(R0 + r, c0 + 64 hf + 16 q4 + c) -= D2[r][64 hf + 16 q4 + c], r = m2
    const int r = m2;
    const bool rok = r < hp;
    const int eYr = eYs[r];
    long long* xr = a.X + R0 + r;
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      if (ok) ok = mbar_wait(smem_u32(acc2), hf, abort, a.st, 9123);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      if (hf == 0 && upper) {
        // half 0's products have read the W buffer: the upper half goes in
        put_digits<S, 8, OZ_BN>(smem + P2_W + q4 * B_KS, m2 - 64, 0, T);
        put_digits<S, 8, OZ_BN>(smem + P2_W + q4 * B_KS, m2 - 64, 8, T + 8);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(fullW));
      }
      tc_fence_after();
      drain16<S, BB_G>(tmem, quad, q4, Rh, Rl);
      tc_fence_before();
      __syncwarp();
      if (hf == 0 && lane == 0) mbar_arrive(smem_u32(drained));
      // D2 = R 2^(eW_c + eY_r - 8S - 6), on the grid 2^(1 - 8S) rounded once:
      // delta = round(R 2^-k), k = 7 - eW_c - eY_r; zero for a zero column of W or a
      // zero row of Y (the padding row h of the tile among them)
      const int cb = 64 * hf + 16 * q4;
      bool fast = true;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int k = 7 - eWs[cb + c] - eYr;
        const bool zero = eWs[cb + c] == -1022 || eYr == -1022;
        fast &= zero | ((k > 0) & (k < G));
      }
      if (__all_sync(0xffffffffu, fast)) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const bool zero = eWs[cb + c] == -1022 || eYr == -1022;
          const long long t = round_split<G>(Rh[c], Rl[c], zero ? 1 : 7 - eWs[cb + c] - eYr);
          Rh[c] = zero ? 0ll : t;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          long long hi;
          unsigned long long lo;
          sum128<S>(Rh[c], Rl[c], hi, lo);
          Rh[c] = round_shift(hi, lo, eWs[cb + c] + eYr - 7);
        }
      }
      long long* xc2 = xr + (c0 + cb) * a.ldx;
      const int64_t left = a.n - (c0 + cb);
      const int ncol = left < 16 ? (int)left : 16;
      if (rok) {
#pragma unroll
        for (int c0r = 0; c0r < 16; c0r += 8) {
          long long cv[8];  // the 8 loads go out before any store
#pragma unroll
          for (int q = 0; q < 8; ++q) cv[q] = (c0r + q < ncol) ? xc2[(c0r + q) * a.ldx] : 0ll;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (c0r + q < ncol) xc2[(c0r + q) * a.ldx] = cv[q] - Rh[c0r + q];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

template <int S>
size_t wave_smem_bytes() {
  constexpr uint32_t A_KS = S * OZ_BM * OZ_KS * 2, B_KS = S * OZ_BN * OZ_KS * 2;
  constexpr uint32_t P1X = BB_P1_STAGES * (A_KS + B_KS) + BB_NX * BB_XS, P2 = 4 * A_KS + 4 * B_KS;
  return 1024 + (P1X > P2 ? P1X : P2) + (14 + 2 * BB_NX) * 8 + 16 + (BB_G + BB_H + 5 * BB_H) * 4 + 64;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the
// driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Buffers of the prepared groups of one chunk: the slices and scales the waves read
// (Vb, Yb, eV, eY, kept until the chunk's waves have run), the FP64 factors and the
// products' scratch.
struct PrepBufs {
  __half* Vb = nullptr;
  __half* Yb = nullptr;
  int* eV = nullptr;
  int* eY = nullptr;
  double* Vg = nullptr;
  double* Yg = nullptr;
  double* Gg = nullptr;
  double* Tg = nullptr;
  double* taug = nullptr;
  char* scratch = nullptr;
  size_t bytes = 0;  // total, the products' scratch included
};

PrepBufs carve_prep(void* base, int count, int ref_slices) {
  Carver cv(base);
  PrepBufs b;
  b.Vb = cv.take<__half>((size_t)count * BB_MAXS * BB_G * BB_H);  // room for the most digits
  b.Yb = cv.take<__half>((size_t)count * BB_MAXS * BB_H * BB_G);
  b.eV = cv.take<int>((size_t)count * BB_G);
  b.eY = cv.take<int>((size_t)count * BB_H);
  b.Vg = cv.take<double>((size_t)count * BB_H * BB_G);
  b.Yg = cv.take<double>((size_t)count * BB_H * BB_G);
  b.Gg = cv.take<double>((size_t)count * BB_G * BB_G);
  b.Tg = cv.take<double>((size_t)count * BB_G * BB_G);
  b.taug = cv.take<double>((size_t)count * BB_G);
  b.scratch = cv.take<char>(0);
  const size_t prod = std::max(ozaki_scratch_bytes_batched(BB_G, BB_G, BB_H, ref_slices, count),
                               ozaki_scratch_bytes_batched(BB_H, BB_G, BB_G, ref_slices, count));
  b.bytes = cv.off + prod + 256;
  return b;
}

// The compact WY factors of `count` groups ((J, k) in gjk) and their slices, in a
// handful of batched launches (the prep of a whole chunk of waves at once).
template <int S>
evd_status_t prep_groups(const PlanCore& pc, const BcWork& bw, const int2* gjk, int count, const PrepBufs& pb,
                         cudaStream_t s) {
  const int64_t n = pc.n;
  const int b = pc.b;
  StatScope sc("bc_back_prep", s);
  k_bb_gather<<<(unsigned)count, 256, 0, s>>>(bw.U, bw.Utau, n, b, gjk, pb.Vg, pb.taug); count_launch();
  EVD_CUDA_TRY(cudaGetLastError());
  const size_t prod_bytes = pb.bytes - (size_t)(pb.scratch - reinterpret_cast<char*>(pb.Vb));
  // G_p = V_p^T V_p
  Gemm gg;
  gg.status = pc.status; gg.tag = "bc_back_prep";
  gg.ta = 'T'; gg.m = BB_G; gg.n = BB_G; gg.k = BB_H; gg.A = pb.Vg; gg.lda = BB_H; gg.B = pb.Vg; gg.ldb = BB_H;
  gg.C = pb.Gg; gg.ldc = BB_G; gg.alpha = 1.0; gg.beta = 0.0;
  Batch bt;
  bt.count = count; bt.sA = (int64_t)BB_H * BB_G; bt.sB = (int64_t)BB_H * BB_G; bt.sC = (int64_t)BB_G * BB_G;
  evd_status_t st = ozaki_gemm_batched(gg, bt, pc.ref_slices, pb.scratch, prod_bytes, s);
  if (st != EVD_OK) return st;
  const size_t tsmem = 2 * (size_t)BB_G * BB_G * sizeof(double);
  st = ensure_dynamic_smem((const void*)k_bb_T, tsmem);
  if (st != EVD_OK) return st;
  k_bb_T<<<(unsigned)count, BB_G, tsmem, s>>>(pb.Gg, pb.taug, pb.Tg); count_launch();
  EVD_CUDA_TRY(cudaGetLastError());
  // Y_p = V_p T_p
  Gemm gy;
  gy.status = pc.status; gy.tag = "bc_back_prep";
  gy.m = BB_H; gy.n = BB_G; gy.k = BB_G; gy.A = pb.Vg; gy.lda = BB_H; gy.B = pb.Tg; gy.ldb = BB_G;
  gy.C = pb.Yg; gy.ldc = BB_H; gy.alpha = 1.0; gy.beta = 0.0;
  bt.sA = (int64_t)BB_H * BB_G; bt.sB = (int64_t)BB_G * BB_G; bt.sC = (int64_t)BB_H * BB_G;
  st = ozaki_gemm_batched(gy, bt, pc.ref_slices, pb.scratch, prod_bytes, s);
  if (st != EVD_OK) return st;
  k_bb_split<S><<<(unsigned)count, 256, 0, s>>>(pb.Vg, pb.Yg, pb.Vb, pb.eV, pb.Yb, pb.eY); count_launch();
  EVD_CUDA_TRY(cudaGetLastError());
  return EVD_OK;
}

// One fused wave over `count` prepared groups starting at group g_off of the chunk.
template <int S>
evd_status_t launch_wave(const PlanCore& pc, double* Q, int64_t ldq, const PrepBufs& pb, int g_off, int count,
                         int64_t R0, int hh0, const WaveTiles& wt, cudaStream_t s) {
  const int64_t n = pc.n;
  const int b = pc.b;
  const size_t smem = wave_smem_bytes<S>();
  evd_status_t st = ensure_dynamic_smem((const void*)k_bcback_wave<S>, smem);
  if (st != EVD_OK) return st;
  WaveArgs a;
  {
    // X (n x n int64, column stride ldq) for the tensor copies of phase 1
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return EVD_ERR_CUDA;
    const cuuint64_t gdim[2] = {(cuuint64_t)n, (cuuint64_t)n};
    const cuuint64_t gstride[1] = {(cuuint64_t)ldq * 8};
    const cuuint32_t box[2] = {(cuuint32_t)BB_XROWS, (cuuint32_t)OZ_BM};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&a.xmap, CU_TENSOR_MAP_DATA_TYPE_INT64, 2, Q, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return EVD_ERR_CUDA;
  }
  a.X = reinterpret_cast<long long*>(Q); a.ldx = ldq; a.n = n; a.R0 = R0; a.gstride = 2 * b; a.h0 = hh0;
  a.h = 2 * b - 1;
  a.Vb = pb.Vb + (size_t)g_off * S * BB_G * BB_H;
  a.eV = pb.eV + (size_t)g_off * BB_G;
  a.Yb = pb.Yb + (size_t)g_off * S * BB_H * BB_G;
  a.eY = pb.eY + (size_t)g_off * BB_H;
  a.st = pc.status;
  a.tile0 = wt.ranges ? wt.tile0 : 0;
  a.ranges = wt.ranges;
  const int64_t ntiles = wt.ranges ? wt.tile1 - wt.tile0 + 1 : ceil_div(n, OZ_BM);
  if (ntiles <= 0) return EVD_OK;
  dim3 grid((unsigned)ntiles, (unsigned)count);
  // executed tile work (the tiles of the range table, when there is one)
  const double tiles = wt.ranges ? (double)wt.work_tiles : (double)count * ceil_div(n, OZ_BM);
  const double flops = tiles * OZ_BM * 2.0 * (BB_G * BB_H + BB_H * BB_G) * (double)(S * (S + 1) / 2);
  StatScope sc("bc_back_wave", s, flops, tiles * 16.0 * BB_H * (double)OZ_BM, "tc_split");
  k_bcback_wave<S><<<grid, BB_THREADS, smem, s>>>(a);
  count_launch();
  EVD_CUDA_TRY(cudaGetLastError());
  return EVD_OK;
}

// X (FP64, in place) <-> fixed point T = round_half_away(x 2^(8S - 1)) (int64).
template <int S>
__global__ void k_x_fixed(double* Q, int64_t ldq, int64_t n, int to_fixed) {
  const int64_t j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double* p = Q + i + j * ldq;
    if (to_fixed) {
      const double x = *p;
      const long long T = scaled_pow2(x, 8 * S - 1);
      *reinterpret_cast<long long*>(p) = T;
    } else {
      const long long T = *reinterpret_cast<const long long*>(p);
      *p = (double)T * (1.0 / (double)(1ll << (8 * S - 1)));
    }
  }
}

template <int S>
evd_status_t fixed_point(double* Q, int64_t ldq, int64_t n, bool to_fixed, cudaStream_t s) {
  for (int64_t j0 = 0; j0 < n; j0 += 65535) {
    const int64_t cols = std::min<int64_t>(n - j0, 65535);
    k_x_fixed<S><<<dim3((unsigned)std::min<int64_t>(ceil_div(n, 256), 16), (unsigned)cols), 256, 0, s>>>(
        Q + j0 * ldq, ldq, n, to_fixed ? 1 : 0);
    count_launch();
  }
  EVD_CUDA_TRY(cudaGetLastError());
  return EVD_OK;
}

}  // namespace

// The fused waves run with 7 digits (55 bits) in both precisions.  A 6-digit build
// gave run-to-run differences in split precision at n = 16384 until the proxy fence
// before an X box is released; with it, repeated solves agree bit for bit, but the
// 6-digit build is not validated at full size and is not instantiated.
constexpr int kWaveDigits = 7;

evd_status_t bcback_fixed_point(const PlanCore& pc, double* Q, int64_t ldq, bool to_fixed) {
  StatScope sc("bc_back_prep", pc.stream);
  return fixed_point<kWaveDigits>(Q, ldq, pc.n, to_fixed, pc.stream);
}

bool bcback_fused_supported(const PlanCore& pc, const double* Q, int64_t ldq) {
  // the tensor copies of X want a 16-byte aligned base and column stride
  return pc.b == BB_G && (pc.slices == 8 || pc.slices == 6) && pc.n >= 1024 && pc.n < ((int64_t)1 << 31) &&
         ldq % 2 == 0 && (reinterpret_cast<uintptr_t>(Q) & 15) == 0;
}

size_t bcback_prep_bytes(int count, int ref_slices) { return carve_prep(nullptr, count, ref_slices).bytes; }

evd_status_t bcback_prep_chunk(const PlanCore& pc, const BcWork& bw, const int2* gjk, int count, void* buf) {
  const PrepBufs pb = carve_prep(buf, count, pc.ref_slices);
  return prep_groups<kWaveDigits>(pc, bw, gjk, count, pb, pc.stream);
}

evd_status_t bcback_fused_wave(const PlanCore& pc, double* Q, int64_t ldq, void* buf, int chunk_count, int g_off,
                               int count, int64_t R0, int hh0, const WaveTiles& wt) {
  const PrepBufs pb = carve_prep(buf, chunk_count, pc.ref_slices);
  return launch_wave<kWaveDigits>(pc, Q, ldq, pb, g_off, count, R0, hh0, wt, pc.stream);
}

size_t bcback_fused_scratch_bytes(int64_t n, int b, int ref_slices) {
  // the prep of a chunk of up to 4096 groups (at least the largest wave)
  const int64_t groups = bc_num_groups(n, b);
  const int chunk = (int)std::max<int64_t>(std::min<int64_t>(groups, 4096), bc_wave_max_groups(n, b));
  return bcback_prep_bytes(chunk, ref_slices) + 256;
}

}  // namespace evd
