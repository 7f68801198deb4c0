// Small device utilities: finiteness check, copies, identity.
#include <cstdio>
#include <map>
#include <mutex>

#include "device_util.cuh"
#include "evd_internal.h"

namespace evd {

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (never lowers
// it: launches of other problem sizes, possibly from other threads, may still rely
// on the larger value).
evd_status_t ensure_dynamic_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<const void*, size_t> set;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set[func];
  if (bytes <= cur) return EVD_OK;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)");
  cur = bytes;
  return EVD_OK;
}

evd_status_t ws_fail(const char* where, size_t have, size_t need) {
  if (getenv("EVD_DEBUG")) fprintf(stderr, "libevd: workspace too small in %s: %zu bytes, %zu needed\n", where, have, need);
  return EVD_ERR_WORKSPACE;
}

evd_status_t cuda_fail(cudaError_t e, const char* what) {
  if (getenv("EVD_DEBUG")) fprintf(stderr, "libevd: %s failed: %s\n", what, cudaGetErrorString(e));
  (void)cudaGetLastError();
  return EVD_ERR_CUDA;
}

__global__ void k_check_finite_lower(const double* __restrict__ A, int64_t lda, int64_t n, int* st) {
  int64_t j = blockIdx.y;
  for (int64_t i = j + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = A[i + j * lda];
    if (!isfinite(v)) {
      dev_set_status(st, EVD_ERR_NONFINITE, (int)(i + 1));
      return;
    }
  }
}

evd_status_t check_finite_lower(const PlanCore& pc, const double* A, int64_t lda) {
  if (pc.n == 0) return EVD_OK;
  for (int64_t j0 = 0; j0 < pc.n; j0 += 65535) {
    int64_t cols = pc.n - j0 < 65535 ? pc.n - j0 : 65535;
    dim3 grid(4, (unsigned)cols);
    k_check_finite_lower<<<grid, 256, 0, pc.stream>>>(A + j0 * lda + j0, lda, pc.n - j0, pc.status); count_launch();
  }
  EVD_CUDA_TRY(cudaGetLastError());
  return EVD_OK;
}

__global__ void k_copy_lower_to_full(const double* __restrict__ A, int64_t lda, double* __restrict__ B,
                                     int64_t ldb, int64_t n) {
  int64_t j = blockIdx.y * 32 + threadIdx.y;
  int64_t i = blockIdx.x * 32 + threadIdx.x;
  if (i < n && j < n) {
    double v = (i >= j) ? A[i + j * lda] : A[j + i * lda];
    B[i + j * ldb] = v;
  }
}

evd_status_t copy_lower_to_full(const double* A, int64_t lda, double* B, int64_t ldb, int64_t n,
                                cudaStream_t s) {
  if (n == 0) return EVD_OK;
  dim3 grid((unsigned)ceil_div(n, 32), (unsigned)ceil_div(n, 32));
  k_copy_lower_to_full<<<grid, dim3(32, 32), 0, s>>>(A, lda, B, ldb, n); count_launch();
  EVD_CUDA_TRY(cudaGetLastError());
  return EVD_OK;
}

evd_status_t copy_matrix(const double* A, int64_t lda, double* B, int64_t ldb, int64_t m, int64_t n,
                         cudaStream_t s) {
  if (m == 0 || n == 0) return EVD_OK;
  EVD_CUDA_TRY(cudaMemcpy2DAsync(B, ldb * sizeof(double), A, lda * sizeof(double), m * sizeof(double), n,
                                 cudaMemcpyDeviceToDevice, s));
  return EVD_OK;
}

__global__ void k_set_identity(double* Q, int64_t ldq, int64_t n, int64_t j0) {
  int64_t j = j0 + blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Q[i + j * ldq] = (i == j) ? 1.0 : 0.0;
}

evd_status_t set_identity(double* Q, int64_t ldq, int64_t n, cudaStream_t s) {
  for (int64_t j0 = 0; j0 < n; j0 += 65535) {
    int64_t cols = n - j0 < 65535 ? n - j0 : 65535;
    k_set_identity<<<dim3(4, (unsigned)cols), 256, 0, s>>>(Q, ldq, n, j0); count_launch();
  }
  EVD_CUDA_TRY(cudaGetLastError());
  return EVD_OK;
}

int max_coresident_blocks(const void* kernel, int threads, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  return per * sms;
}

}  // namespace evd
