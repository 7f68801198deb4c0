// Self-test of the bounded device waits.  Every wait in the library (progress
// flags, grid barriers, mbarriers) gives up after a limit, latches EVD_ERR_TIMEOUT
// with a location code in the plan's status word, and lets its kernel return, so
// that the context stays usable.  evd_wait_selftest runs one such wait on
// something that never completes -- a flag nothing publishes, a barrier that
// counts one arrival more than the grid has CTAs, an mbarrier nobody arrives at --
// with a short limit, through the same helpers the solver uses.
#include "device_util.cuh"
#include "evd_internal.h"
#include "tc_common.cuh"

namespace evd {
namespace {

constexpr long long kTestLimit = 1 << 16;  // polls: well under a second

// kind 0: progress-flag wait on a flag that stays 0.
__global__ void k_selftest_flag(const int* flag, int* st) {
  if (threadIdx.x == 0) wait_geq(flag, 1, st, 9901, kTestLimit);
}

// kind 1: grid barrier expecting one CTA more than the launch has.
__global__ void k_selftest_barrier(unsigned* bar, int* st) {
  grid_barrier(bar, gridDim.x + 1, st, 9902, kTestLimit);
}

// kind 2: a CTA that holds tensor memory waits on an mbarrier nobody arrives at,
// gives up, frees its tensor memory and returns.
__global__ void k_selftest_mbarrier(int* st) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    tcx::mbar_init(tcx::smem_u32(&bar), 1);
    abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(tcx::smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  tcx::tc_fence_after();
  if (threadIdx.x == 32)
    tcx::mbar_wait(tcx::smem_u32(&bar), 0, reinterpret_cast<volatile int*>(&abort), st, 9903, kTestLimit);
  tcx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tcx::tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem_slot) : "memory");
  }
}

}  // namespace

evd_status_t wait_selftest(const PlanCore& pc, int kind, int* flag_zero, unsigned* bar) {
  cudaStream_t s = pc.stream;
  switch (kind) {
    case 0:
      EVD_CUDA_TRY(cudaMemsetAsync(flag_zero, 0, sizeof(int), s));
      k_selftest_flag<<<1, 32, 0, s>>>(flag_zero, pc.status);
      break;
    case 1:
      k_selftest_barrier<<<1, 64, 0, s>>>(bar, pc.status);
      break;
    case 2:
      k_selftest_mbarrier<<<1, 64, 0, s>>>(pc.status);
      break;
    default:
      return EVD_ERR_INVALID_ARG;
  }
  count_launch();
  EVD_CUDA_TRY(cudaGetLastError());
  return EVD_OK;
}

}  // namespace evd
