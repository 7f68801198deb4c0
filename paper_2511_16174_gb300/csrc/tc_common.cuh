// Shared device code of the tensor-core split products: slice layout, digit
// extraction, the PTX wrappers (mbarrier, bulk copy, tcgen05), the unrolled issue of
// one K-step's slice-pair products, and the exact 128-bit to FP64 conversion.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "device_util.cuh"

namespace evd {
namespace tcx {

constexpr int OZ_BM = 128;        // tile rows (tensor-memory lanes)
constexpr int OZ_BN = 64;         // tile columns (per weight accumulator)
constexpr int OZ_KS = 16;         // K-elements per MMA K-step
constexpr int OZ_MAXS = 8;        // slices
constexpr long long OZ_WAIT_LIMIT = 1ll << 26;

// Element index of (row R, K-element k) of slice t in the blob layout with TR-row
// tiles and nkb K-blocks per row tile (R counts rows over all batched problems).
__device__ __forceinline__ size_t blob_index(int64_t R, int64_t k, int t, int s, int TR, int64_t nkb) {
  const int64_t tile = R / TR, rr = R - tile * TR, kb = k >> 4, kk = k & 15;
  return ((size_t)(tile * nkb + kb) * s + t) * (size_t)(TR * 16) + (size_t)(((rr >> 3) * 2 + (kk >> 3)) * 64) +
         (size_t)((rr & 7) * 8 + (kk & 7));
}

// T = round_half_away(x 2^(7s - e)), the scaled operand as an integer.
__device__ __forceinline__ long long ozaki_scaled(double x, int e, int s) {
  const long long bits = __double_as_longlong(x);
  int E = (int)((bits >> 52) & 0x7FF);
  long long m = bits & 0xFFFFFFFFFFFFFll;
  long long T = 0;
  if (E != 0 || m != 0) {
    if (E == 0) E = 1; else m |= (1ll << 52);
    const int sh = E - 1075 + 7 * s - e;  // |x| = m 2^(E - 1075);  T = m 2^sh
    if (sh >= 0) T = m << sh;
    else {
      const int r = -sh;
      T = (r >= 63) ? 0 : ((m + (1ll << (r - 1))) >> r);
    }
    if (bits < 0) T = -T;
  }
  return T;
}

// Balanced base-128 digits, each on its own: with the offset
// O = 64 (1 + 128 + ... + 128^(s-2)), the low s-1 balanced digits of T are the
// ordinary base-128 digits of T + O minus 64, and the top digit is (T + O) >> 7(s-1).
// Slice t holds the digit at position s-1-t (slice 0 is the top).
__device__ __forceinline__ long long ozaki_offset(int s) {
  long long o = 0;
  for (int j = 0; j < s - 1; ++j) o = (o << 7) + 64;
  return o;
}
__device__ __forceinline__ int ozaki_digit(long long TO, int s, int t) {
  const int j = s - 1 - t;
  return (t == 0) ? (int)(TO >> (7 * j)) : (int)((TO >> (7 * j)) & 127) - 64;
}

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait (`limit` polls); raises *abort (shared) and the status word on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort, int* st, int where,
                                          long long limit = OZ_WAIT_LIMIT) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try(a, parity)) return true;
    if (*abort) return false;
  }
  *abort = 1;
  dev_set_status(st, EVD_ERR_TIMEOUT, where);
  return false;
}
// Contiguous global -> shared bulk copy completing on an mbarrier (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
// K-major operand without swizzle: core matrices of 8 rows x 16 bytes stored as
// 128 contiguous bytes; the two core matrices of a 16-element K step are 128 bytes
// apart (leading byte offset), consecutive 8-row groups 256 bytes apart (stride
// byte offset).
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;    // leading byte offset: next core matrix along K
  d |= (uint64_t)(256 >> 4) << 32;    // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;             // descriptor version (sm_100 family)
  return d;                           // layout type 0: no swizzle
}
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x 2^ex as a double, rounded to nearest even, from the signed 128-bit integer
// (hi, lo) -- integer operations only (GB300's FP64 pipe is narrow).  Falls back to
// FP64 arithmetic only when the result is subnormal or overflows.
__device__ __forceinline__ double i128_to_double(long long hi, unsigned long long lo, int ex) {
  const bool neg = hi < 0;
  unsigned long long mh = (unsigned long long)hi, ml = lo;
  if (neg) {  // two's complement negate
    ml = ~ml + 1ull;
    mh = ~mh + (ml == 0ull ? 1ull : 0ull);
  }
  if (mh == 0ull && ml == 0ull) return 0.0;
  // position of the top bit
  int p;
  if (mh != 0ull) p = 127 - __clzll((long long)mh);
  else p = 63 - __clzll((long long)ml);
  unsigned long long m;
  int E = p + ex;  // value = 1.xxx * 2^E
  if (p <= 52) {
    m = ml << (52 - p);
  } else {
    const int sh = p - 52;  // bits dropped below the 53-bit mantissa
    // m = (mh:ml) >> sh, sticky and round bits
    unsigned long long q;
    if (sh < 64) {
      q = (ml >> sh) | (sh ? (mh << (64 - sh)) : 0ull);
      const unsigned long long rem_lo = sh ? (ml << (64 - sh)) : 0ull;  // dropped bits, left-aligned
      const unsigned long long half = 1ull << 63;
      const bool round_up = (rem_lo > half) || (rem_lo == half && (q & 1ull));
      m = q + (round_up ? 1ull : 0ull);
    } else {
      const int s2 = sh - 64;
      q = mh >> s2;
      // dropped bits, left-aligned in (d_hi, d_lo)
      const unsigned long long d_hi = s2 ? ((mh << (64 - s2)) | (ml >> s2)) : ml;
      const unsigned long long d_lo = s2 ? (ml << (64 - s2)) : 0ull;
      const unsigned long long half = 1ull << 63;
      const bool above = (d_hi > half) || (d_hi == half && d_lo != 0ull);
      const bool tie = (d_hi == half && d_lo == 0ull);
      const bool round_up = above || (tie && (q & 1ull));
      m = q + (round_up ? 1ull : 0ull);
    }
    if (m >> 53) { m >>= 1; ++E; }
  }
  const int biased = E + 1023;
  if (biased <= 0 || biased >= 2047) {
    // rare: finish in FP64 arithmetic
    double v = ldexp((double)(m & ((1ull << 53) - 1)), E - 52);
    return neg ? -v : v;
  }
  const unsigned long long bits = ((unsigned long long)neg << 63) | ((unsigned long long)biased << 52) |
                                  (m & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

// All slice-pair products of one K-step for S slices: for each A slice t, the B
// slices u = 0 .. S-1-t in groups of up to four stacked along N (N <= 256), into the
// weight accumulators t+u0 .. at TMEM columns 64 (t + u0).  Fully unrolled: every
// descriptor is the stage's base descriptor plus a constant (the 14-bit address
// field cannot carry: shared-memory addresses stay below 2^18 bytes).  The first
// products into each weight (t = 0) take acc_t0 (0 at the start of a drain chunk).
// F16: both operands float16 (the fused BC-Back waves' 8-bit digits) instead of
// bfloat16.
template <int S, bool F16 = false>
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint64_t da0, uint64_t db0, uint32_t acc_t0) {
  constexpr uint32_t kFmt = F16 ? 0u : (1u << 7) | (1u << 10);  // A and B format: 0 float16, 1 bfloat16
  constexpr uint32_t kIdesc = (1u << 4) | kFmt | ((uint32_t)(OZ_BM >> 4) << 24);
#pragma unroll
  for (int t = 0; t < S; ++t) {
#pragma unroll
    for (int u0 = 0; u0 < S - t; u0 += 4) {
      const int cnt = (S - t - u0 < 4) ? S - t - u0 : 4;
      tc_mma(tmem + (uint32_t)((t + u0) * OZ_BN), da0 + (uint64_t)((t * OZ_BM * OZ_KS * 2) >> 4),
             db0 + (uint64_t)((u0 * OZ_BN * OZ_KS * 2) >> 4),
             kIdesc | ((uint32_t)((OZ_BN * cnt) >> 3) << 17), t == 0 ? acc_t0 : 1u);
    }
  }
}

}  // namespace tcx
}  // namespace evd
