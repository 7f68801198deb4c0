// Batched solves and the (b, nb) autotuner.
//
// Batched: problems are assigned longest-processing-time first (cost ~ n^3) to up
// to kMaxLanes "lanes".  Each lane is a CUDA stream of its own, driven by a host
// thread of its own, with its own slice of the caller's workspace; lanes start
// after the caller's stream reaches the call and the caller's stream waits for
// every lane at the end.  Within a lane the problems run one after another with a
// plan each (the divide-and-conquer stage reads its deflation counts on the host,
// so a lane's host thread waits at those points while the other lanes keep the GPU
// busy).
//
// Autotuner: times candidate (b, nb) pairs on a seeded symmetric matrix of the
// requested order and keeps the fastest per (n bucket, job, precision) in a JSON
// cache file of one entry per line.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "evd_internal.h"

namespace evd {
namespace {

constexpr int kMaxLanes = 8;

struct Assignment {
  int lanes = 0;
  std::vector<std::vector<int>> items;  // problem indices per lane, longest first
  std::vector<size_t> ws_bytes;         // workspace per lane
  std::vector<size_t> ws_offset;        // 256-byte aligned offsets into the caller's workspace
  size_t total = 0;
};

size_t plan_ws_bytes(int64_t n, int64_t lda, evd_job_t job, evd_status_t* st) {
  *st = (n >= 0 && lda >= std::max<int64_t>(1, n) && n < ((int64_t)1 << 31)) ? EVD_OK : EVD_ERR_INVALID_ARG;
  return (*st == EVD_OK) ? plan_workspace_bytes(n, lda, job, EVD_FP64, 0, 0) : 0;
}

// Longest processing time first: sort by n descending, give each problem to the
// lane with the least assigned n^3 so far.
evd_status_t assign(int count, const int64_t* n, const int64_t* lda, evd_job_t job, Assignment* out) {
  Assignment a;
  a.lanes = std::min(count, kMaxLanes);
  a.items.assign(a.lanes, {});
  a.ws_bytes.assign(a.lanes, 256);
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return n[x] > n[y]; });
  std::vector<double> load(a.lanes, 0.0);
  for (int i : order) {
    const int lane = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[lane] += (double)n[i] * (double)n[i] * (double)n[i] + 1.0;
    a.items[lane].push_back(i);
    evd_status_t st;
    const size_t b = plan_ws_bytes(n[i], lda ? lda[i] : std::max<int64_t>(n[i], 1), job, &st);
    if (st != EVD_OK) return st;
    a.ws_bytes[lane] = std::max(a.ws_bytes[lane], b);
  }
  a.ws_offset.assign(a.lanes, 0);
  size_t off = 0;
  for (int l = 0; l < a.lanes; ++l) {
    a.ws_offset[l] = off;
    off = align_up(off + a.ws_bytes[l], 256);
  }
  a.total = std::max<size_t>(off, 256);
  *out = std::move(a);
  return EVD_OK;
}

// ---------------------------------------------------------------- autotuner
__global__ void k_fill_symmetric(double* A, int64_t n, uint64_t seed) {
  const int64_t j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t lo = (uint64_t)(i < j ? i : j), hi = (uint64_t)(i < j ? j : i);
    uint64_t x = seed ^ (hi * 0x9E3779B97F4A7C15ull) ^ (lo * 0xC2B2AE3D27D4EB4Full);
    x ^= x >> 33; x *= 0xFF51AFD7ED558CCDull; x ^= x >> 33; x *= 0xC4CEB9FE1A85EC53ull; x ^= x >> 33;
    A[i + j * n] = (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;  // uniform in [-1, 1)
  }
}

int64_t bucket_of(int64_t n) {
  if (n <= 1) return 1;
  const double l = std::log2((double)n);
  return (int64_t)1 << (int)std::lround(l);
}

struct CacheEntry {
  int64_t bucket;
  int job, prec, b, nb;
  double ms;
};

std::mutex g_cache_mu;

std::vector<CacheEntry> read_cache(const char* path) {
  std::vector<CacheEntry> v;
  if (!path) return v;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    CacheEntry e{};
    long long bk = 0;
    if (sscanf(line.c_str(), " {\"n_bucket\": %lld, \"job\": %d, \"prec\": %d, \"b\": %d, \"nb\": %d, \"ms\": %lf",
               &bk, &e.job, &e.prec, &e.b, &e.nb, &e.ms) == 6) {
      e.bucket = bk;
      v.push_back(e);
    }
  }
  return v;
}

void write_cache(const char* path, const std::vector<CacheEntry>& v) {
  if (!path) return;
  std::ofstream f(path, std::ios::trunc);
  f << "[\n";
  for (size_t i = 0; i < v.size(); ++i) {
    char buf[256];
    snprintf(buf, sizeof(buf), "{\"n_bucket\": %lld, \"job\": %d, \"prec\": %d, \"b\": %d, \"nb\": %d, \"ms\": %.3f}%s\n",
             (long long)v[i].bucket, v[i].job, v[i].prec, v[i].b, v[i].nb, v[i].ms, i + 1 < v.size() ? "," : "");
    f << buf;
  }
  f << "]\n";
}

}  // namespace

// Cached choice for plan creation with b = nb = 0 (no timing): the entry of the
// file named by EVD_AUTOTUNE_CACHE for n's bucket, job and precision, if any.
bool autotune_lookup(int64_t n, evd_job_t job, evd_prec_t prec, int* b, int* nb) {
  const char* path = getenv("EVD_AUTOTUNE_CACHE");
  if (!path) return false;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  for (const CacheEntry& e : read_cache(path))
    if (e.bucket == bucket_of(n) && e.job == (int)job && e.prec == (int)prec) {
      *b = e.b;
      *nb = e.nb;
      return true;
    }
  return false;
}

}  // namespace evd

using namespace evd;

extern "C" {

evd_status_t evd_batched_workspace_size(int count, const int64_t* n_host, evd_job_t job, size_t* bytes) {
  if (count < 0 || !bytes || (count > 0 && !n_host)) return EVD_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (n_host[i] < 0) return EVD_ERR_INVALID_ARG;
  if (count == 0) { *bytes = 256; return EVD_OK; }
  Assignment a;
  evd_status_t st = assign(count, n_host, nullptr, job, &a);
  if (st != EVD_OK) return st;
  *bytes = a.total;
  return EVD_OK;
}

evd_status_t evd_syevd_batched(int count, const int64_t* n_host, double* const* A_host, const int64_t* lda_host,
                               double* const* w_host, double* const* Q_host, const int64_t* ldq_host, evd_job_t job,
                               void* ws, size_t ws_bytes, void* stream) {
  if (count < 0 || (count > 0 && (!n_host || !A_host || !lda_host || !w_host))) return EVD_ERR_INVALID_ARG;
  if (job == EVD_VECTORS && count > 0 && (!Q_host || !ldq_host)) return EVD_ERR_INVALID_ARG;
  if (count == 0) return EVD_OK;
  for (int i = 0; i < count; ++i)
    if (n_host[i] < 0 || lda_host[i] < std::max<int64_t>(1, n_host[i])) return EVD_ERR_INVALID_ARG;
  Assignment a;
  evd_status_t st = assign(count, n_host, nullptr, job, &a);
  if (st != EVD_OK) return st;
  if (!ws || ws_bytes < a.total || reinterpret_cast<uintptr_t>(ws) % 256 != 0) return EVD_ERR_WORKSPACE;
  int dev = 0;
  EVD_CUDA_TRY(cudaGetDevice(&dev));
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  std::vector<cudaStream_t> lanes(a.lanes, nullptr);
  std::vector<cudaEvent_t> done(a.lanes, nullptr);
  cudaEvent_t start = nullptr;
  auto cleanup = [&]() {
    for (auto& e : done) if (e) cudaEventDestroy(e);
    for (auto& l : lanes) if (l) cudaStreamDestroy(l);
    if (start) cudaEventDestroy(start);
  };
  if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) { cleanup(); return EVD_ERR_CUDA; }
  for (int l = 0; l < a.lanes; ++l) {
    if (cudaStreamCreateWithFlags(&lanes[l], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&done[l], cudaEventDisableTiming) != cudaSuccess) {
      cleanup();
      return EVD_ERR_CUDA;
    }
  }
  if (cudaEventRecord(start, caller) != cudaSuccess) { cleanup(); return EVD_ERR_CUDA; }
  std::vector<evd_status_t> result(a.lanes, EVD_OK);
  auto worker = [&](int l) {
    if (cudaSetDevice(dev) != cudaSuccess || cudaStreamWaitEvent(lanes[l], start, 0) != cudaSuccess) {
      result[l] = EVD_ERR_CUDA;
      return;
    }
    void* wsl = static_cast<char*>(ws) + a.ws_offset[l];
    for (int i : a.items[l]) {
      evd_plan_t p = nullptr;
      evd_status_t s = evd_plan_create(&p, n_host[i], lda_host[i], job, EVD_FP64, 0, 0, lanes[l]);
      if (s == EVD_OK)
        s = evd_syevd(p, A_host[i], w_host[i], job == EVD_VECTORS ? Q_host[i] : nullptr,
                      job == EVD_VECTORS ? ldq_host[i] : 1, wsl);
      if (s == EVD_OK) {
        int info = 0;
        s = evd_plan_status(p, &info);
      }
      evd_plan_destroy(p);
      if (s != EVD_OK) {
        result[l] = s;
        return;
      }
    }
  };
  std::vector<std::thread> threads;
  for (int l = 1; l < a.lanes; ++l) threads.emplace_back(worker, l);
  worker(0);
  for (auto& t : threads) t.join();
  evd_status_t st_all = EVD_OK;
  for (int l = 0; l < a.lanes; ++l) {
    if (st_all == EVD_OK && result[l] != EVD_OK) st_all = result[l];
    if (cudaEventRecord(done[l], lanes[l]) != cudaSuccess || cudaStreamWaitEvent(caller, done[l], 0) != cudaSuccess)
      st_all = (st_all == EVD_OK) ? EVD_ERR_CUDA : st_all;
  }
  // the lanes' work is complete (each lane's last plan status synchronized it), so
  // the streams can go; destroying a stream with pending work would also be safe
  cleanup();
  return st_all;
}

evd_status_t evd_autotune(int64_t n, evd_job_t job, evd_prec_t prec, const char* cache_path, int* b, int* nb) {
  if (!b || !nb || n < 0) return EVD_ERR_INVALID_ARG;
  if (prec == EVD_SPLIT_INT8) return EVD_ERR_NOT_SUPPORTED;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (const CacheEntry& e : read_cache(cache_path))
      if (e.bucket == bucket_of(n) && e.job == (int)job && e.prec == (int)prec) {
        *b = e.b;
        *nb = e.nb;
        return EVD_OK;
      }
  }
  if (n < 64) {  // nothing to tune: the smallest band
    *b = 32;
    *nb = 32;
    return EVD_OK;
  }
  static const int cand[][2] = {{32, 32}, {32, 64}, {32, 128}, {64, 64}, {64, 128}, {128, 128}};
  double* A = nullptr;
  double* A0 = nullptr;
  double* w = nullptr;
  double* Q = nullptr;
  void* ws = nullptr;
  size_t ws_cap = 0;
  auto release = [&]() {
    if (A) cudaFree(A);
    if (A0) cudaFree(A0);
    if (w) cudaFree(w);
    if (Q) cudaFree(Q);
    if (ws) cudaFree(ws);
  };
  const size_t mat = (size_t)n * (size_t)n * sizeof(double);
  if (cudaMalloc(&A, mat) != cudaSuccess || cudaMalloc(&A0, mat) != cudaSuccess ||
      cudaMalloc(&w, (size_t)n * sizeof(double)) != cudaSuccess ||
      (job == EVD_VECTORS && cudaMalloc(&Q, mat) != cudaSuccess)) {
    release();
    return EVD_ERR_OOM;
  }
  if (n > 65535) { release(); return EVD_ERR_NOT_SUPPORTED; }  // the fill kernel's grid.y = n
  k_fill_symmetric<<<dim3((unsigned)std::min<int64_t>(ceil_div(n, 256), 64), (unsigned)n), 256>>>(A0, n, 16174);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) { release(); return EVD_ERR_CUDA; }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300;
  int bb = 0, bnb = 0;
  evd_status_t err = EVD_OK;
  for (const auto& c : cand) {
    if (c[0] >= n) continue;
    evd_plan_t p = nullptr;
    if (evd_plan_create(&p, n, n, job, prec, c[0], c[1], nullptr) != EVD_OK) continue;
    size_t need = 0;
    evd_plan_workspace_size(p, &need);
    if (need > ws_cap) {
      if (ws) cudaFree(ws);
      ws = nullptr;
      if (cudaMalloc(&ws, need) != cudaSuccess) { evd_plan_destroy(p); err = EVD_ERR_OOM; break; }
      ws_cap = need;
    }
    double ms_c = 0.0;
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {  // one untimed warm-up, one timed solve
      cudaMemcpyAsync(A, A0, mat, cudaMemcpyDeviceToDevice, nullptr);
      cudaEventRecord(e0, nullptr);
      ok = evd_syevd(p, A, w, Q, n, ws) == EVD_OK;
      cudaEventRecord(e1, nullptr);
      int info = 0;
      ok = ok && evd_plan_status(p, &info) == EVD_OK;
      float t = 0;
      cudaEventElapsedTime(&t, e0, e1);
      ms_c = t;
    }
    evd_plan_destroy(p);
    if (ok && ms_c < best) {
      best = ms_c;
      bb = c[0];
      bnb = c[1];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release();
  if (err != EVD_OK) return err;
  if (bb == 0) return EVD_ERR_CUDA;
  *b = bb;
  *nb = bnb;
  if (cache_path) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    std::vector<CacheEntry> v = read_cache(cache_path);
    v.push_back({bucket_of(n), (int)job, (int)prec, bb, bnb, best});
    write_cache(cache_path, v);
  }
  return EVD_OK;
}

}  // extern "C"
