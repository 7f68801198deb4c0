// evd_dgemm_static: the FP64 / split-precision product with its scratch taken from a
// fixed array in device global memory instead of a caller workspace.
//
// Who needs it: callers that cannot allocate device memory or pass a workspace
// through.  Examples are a plain C host that links libevd without any device
// allocator, and a callback with a fixed signature that has no workspace
// argument.  It also serves code that must not call cudaMalloc/cudaFree, because
// those are device-wide operations; cudaFree in particular synchronizes with work
// queued on other streams.  This entry point allocates nothing: no cudaMalloc, no
// cudaFree, no allocating library routine.
//
// Limits and rules:
// * The scratch is EVD_STATIC_SCRATCH_BYTES (64 MiB) per device.  A product whose
//   scratch need (evd_gemm_workspace_size) is larger is rejected with
//   EVD_ERR_WORKSPACE before any device work.
// * Every call shares the one array, so calls that overlap in time race.  This
//   covers calls on different streams and calls from different host threads.
//   Calls queued one after another on the same stream are ordered by that stream
//   and are safe.
// * The device address of the array is looked up once per device, on the first
//   call made with that device current.  That lookup may load the module.  Make the
//   first call on each device outside any stream capture.
#include <mutex>

#include "evd_internal.h"
#include "evd_ozaki.h"

namespace evd {
namespace {

// status word (kStatusWords ints) at the front, product scratch after it
constexpr size_t kStatusBytes = 256;
static __device__ __align__(256) unsigned char g_static_scratch[kStatusBytes + EVD_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned char* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_scratch for the current device (looked up once).
evd_status_t static_scratch(unsigned char** out) {
  int dev = 0;
  EVD_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return EVD_ERR_NOT_SUPPORTED;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                                 "cudaGetSymbolAddress(g_static_scratch)");
    g_static_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_static_ptr[dev];
  return EVD_OK;
}

}  // namespace

// Read and clear the status word at the array's front (the last static call's).
evd_status_t static_status_take(int* code, int* info) {
  *code = 0;
  *info = 0;
  int dev = 0;
  EVD_CUDA_TRY(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (dev >= 0 && dev < kMaxDevices) base = g_static_ptr[dev];
  }
  if (!base) return EVD_OK;  // no static call on this device yet
  int h[kStatusWords] = {0};
  EVD_CUDA_TRY(cudaMemcpy(h, base, sizeof(h), cudaMemcpyDeviceToHost));
  EVD_CUDA_TRY(cudaMemset(base, 0, sizeof(h)));
  *code = h[0];
  *info = h[1];
  return EVD_OK;
}

}  // namespace evd

using namespace evd;

extern "C" {

evd_status_t evd_dgemm_status(void* stream, int* info) {
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    (void)cudaGetLastError();
    return EVD_ERR_CUDA;
  }
  int c1 = 0, i1 = 0, c2 = 0, i2 = 0;
  evd_status_t st = standalone_status_take(&c1, &i1);
  if (st != EVD_OK) return st;
  st = static_status_take(&c2, &i2);
  if (st != EVD_OK) return st;
  if (info) *info = c1 ? i1 : i2;
  return static_cast<evd_status_t>(c1 ? c1 : c2);
}

evd_status_t evd_dgemm_static(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                              const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                              int64_t ldc, int slices, void* stream) {
  transa = (char)toupper(transa);
  transb = (char)toupper(transb);
  if ((transa != 'N' && transa != 'T') || (transb != 'N' && transb != 'T')) return EVD_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0 || slices < 0 || slices > 8) return EVD_ERR_INVALID_ARG;
  const int64_t ar = (transa == 'N') ? m : k, br = (transb == 'N') ? k : n;
  if (lda < (ar > 1 ? ar : 1) || ldb < (br > 1 ? br : 1) || ldc < (m > 1 ? m : 1)) return EVD_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && (!C || (k > 0 && (!A || !B)))) return EVD_ERR_INVALID_ARG;
  // oversize: rejected before touching the device.  The least scratch counts (no
  // K-split): the product lowers its split count to what the array holds.
  if (slices > 0 && ozaki_scratch_bytes_min(m, n, k, slices) > (size_t)EVD_STATIC_SCRATCH_BYTES)
    return EVD_ERR_WORKSPACE;
  if (m == 0 || n == 0) return EVD_OK;
  unsigned char* base = nullptr;
  const evd_status_t st = static_scratch(&base);
  if (st != EVD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the status word must start at zero: a timeout latches into it only when it is 0
  int* status = reinterpret_cast<int*>(base);
  EVD_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int) * kStatusWords, s));
  Gemm g;
  g.ta = transa; g.tb = transb; g.m = m; g.n = n; g.k = k; g.alpha = alpha; g.A = A; g.lda = lda;
  g.B = B; g.ldb = ldb; g.beta = beta; g.C = C; g.ldc = ldc;
  g.force_tc = true;
  g.status = status;
  return gemm(g, slices, base + kStatusBytes, (size_t)EVD_STATIC_SCRATCH_BYTES, s);
}

}  // extern "C"
