// Device helpers: status word, bounded waits, deterministic block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "evd_internal.h"

namespace evd {

// Latch the first error code; record info with it.
__device__ inline void dev_set_status(int* st, int code, int info) {
  if (atomicCAS(st, 0, code) == 0) atomicExch(st + 1, info);
}

__device__ inline int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline unsigned ld_acquire_u(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *flag >= target.  Bounded: after `limit` polls the status word gets
// EVD_ERR_TIMEOUT (info = where) and the function returns false.  Also returns
// false as soon as another CTA has raised the abort flag (status[2]).
__device__ inline bool wait_geq(const int* flag, int target, int* st, int where, long long limit = kSpinLimit) {
  // busy polling first (the waits on the critical path are short), then back off
  for (int it = 0; it < 20000; ++it)
    if (ld_acquire(flag) >= target) return true;
  for (long long it = 0; it < limit; ++it) {
    if (ld_acquire(flag) >= target) return true;
    if (ld_acquire(st + 2) != 0) return false;
    __nanosleep(64);
  }
  dev_set_status(st, EVD_ERR_TIMEOUT, where);
  atomicExch(st + 2, 1);
  return false;
}

// Grid barrier for a cooperative launch (all CTAs co-resident).  bar[0] counts
// arrivals, bar[1] is the generation.  Bounded (`limit` polls); returns false on
// timeout/abort, after which every CTA must return.  A barrier that timed out
// leaves its arrival count behind: evd_plan_status clears it with the status word.
__device__ inline bool grid_barrier(unsigned* bar, unsigned nblocks, int* st, int where,
                                    long long limit = kSpinLimit) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    ok_s = 1;
    unsigned gen = ld_acquire_u(bar + 1);
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      bool done = false;
      for (int q = 0; q < 20000 && !done; ++q) done = (ld_acquire_u(bar + 1) != gen);
      for (; !done && it < limit; ++it) {
        if (ld_acquire_u(bar + 1) != gen) break;
        if (ld_acquire(st + 2) != 0) { ok_s = 0; break; }
        __nanosleep(32);
      }
      if (!done && it == limit) {
        dev_set_status(st, EVD_ERR_TIMEOUT, where);
        atomicExch(st + 2, 1);
        ok_s = 0;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok_s != 0;
}

// Deterministic block sum of one double per thread (fixed tree order).
template <int NT>
__device__ inline double block_sum(double v, double* sh) {
  __syncthreads();
  sh[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace evd
