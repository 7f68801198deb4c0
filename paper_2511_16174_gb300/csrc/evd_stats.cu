// Optional per-category timing (CUDA events on the launching stream), algorithmic
// flop/byte counts and a launch counter, for the benchmark's roofline report.
// Disabled by default; when disabled every hook is one relaxed atomic load.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "evd_internal.h"

namespace evd {

namespace {
struct Rec {
  cudaEvent_t a, b;
};
struct Cat {
  std::vector<Rec> recs;
  double flops = 0, bytes = 0;
  int64_t calls = 0;
};
std::atomic<bool> g_on{false};
std::atomic<int64_t> g_launches{0};
std::mutex g_mu;
std::map<std::string, Cat> g_cats;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
std::string key_of(const char* cat, const char* engine) {
  std::string k(cat ? cat : "");
  if (engine) {
    k += '/';
    k += engine;
  }
  return k;
}
}  // namespace

StatScope::StatScope(const char* cat, cudaStream_t s, double flops, double bytes, const char* engine)
    : cat_(cat), engine_(engine), s_(s) {
  on_ = g_on.load(std::memory_order_relaxed);
  if (!on_) return;
  // no timing events inside a stream capture (a captured solve is timed as a whole)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s_, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    (void)cudaGetLastError();
    on_ = false;
    return;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  a_ = take_event();
  cudaEventRecord(static_cast<cudaEvent_t>(a_), s_);
  Cat& c = g_cats[key_of(cat_, engine_)];
  c.flops += flops;
  c.bytes += bytes;
  c.calls += 1;
}

StatScope::~StatScope() {
  if (!on_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  cudaEventRecord(b, s_);
  g_cats[key_of(cat_, engine_)].recs.push_back({static_cast<cudaEvent_t>(a_), b});
}

}  // namespace evd

using namespace evd;

extern "C" {

void evd_stats_enable(int on) { g_on.store(on != 0); }

void evd_stats_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& kv : g_cats)
    for (auto& r : kv.second.recs) {
      g_pool.push_back(r.a);
      g_pool.push_back(r.b);
    }
  g_cats.clear();
  g_launches.store(0);
}

int64_t evd_launch_count(void) { return g_launches.load(); }

// Category names joined by '\n' into buf (size cap); returns the number of categories.
int evd_stats_categories(char* buf, int cap) {
  std::lock_guard<std::mutex> lk(g_mu);
  std::string s;
  for (auto& kv : g_cats) {
    if (!s.empty()) s += '\n';
    s += kv.first;
  }
  if (buf && cap > 0) {
    strncpy(buf, s.c_str(), (size_t)cap - 1);
    buf[cap - 1] = 0;
  }
  return (int)g_cats.size();
}

// Total device time (ms, sum of per-call event intervals), algorithmic flops and
// bytes, and calls of one category.  Synchronizes the recorded events.
evd_status_t evd_stats_query(const char* cat, double* ms, double* flops, double* bytes, int64_t* calls) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cats.find(cat ? cat : "");
  if (it == g_cats.end()) {
    if (ms) *ms = 0; if (flops) *flops = 0; if (bytes) *bytes = 0; if (calls) *calls = 0;
    return EVD_OK;
  }
  double tot = 0;
  for (auto& r : it->second.recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return EVD_ERR_CUDA;
    float t = 0;
    cudaEventElapsedTime(&t, r.a, r.b);
    tot += t;
  }
  if (ms) *ms = tot;
  if (flops) *flops = it->second.flops;
  if (bytes) *bytes = it->second.bytes;
  if (calls) *calls = it->second.calls;
  return EVD_OK;
}

}  // extern "C"
