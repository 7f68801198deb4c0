// Batched solves and the (b, nb) autotuner.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "evd_internal.h"

extern "C" {

evd_status_t evd_batched_workspace_size(int count, const int64_t* n_host, evd_job_t job, size_t* bytes) {
  if (count < 0 || !bytes || (count > 0 && !n_host)) return EVD_ERR_INVALID_ARG;
  size_t mx = 256;
  for (int i = 0; i < count; ++i) {
    if (n_host[i] < 0) return EVD_ERR_INVALID_ARG;
    evd_plan_t p = nullptr;
    evd_status_t st = evd_plan_create(&p, n_host[i], std::max<int64_t>(n_host[i], 1), job, EVD_FP64, 0, 0, nullptr);
    if (st != EVD_OK) return st;
    size_t b = 0;
    evd_plan_workspace_size(p, &b);
    evd_plan_destroy(p);
    mx = std::max(mx, b);
  }
  *bytes = mx;
  return EVD_OK;
}

evd_status_t evd_syevd_batched(int count, const int64_t* n_host, double* const* A_host, const int64_t* lda_host,
                               double* const* w_host, double* const* Q_host, const int64_t* ldq_host, evd_job_t job,
                               void* ws, size_t ws_bytes, void* stream) {
  if (count < 0 || (count > 0 && (!n_host || !A_host || !lda_host || !w_host))) return EVD_ERR_INVALID_ARG;
  if (job == EVD_VECTORS && count > 0 && (!Q_host || !ldq_host)) return EVD_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    evd_plan_t p = nullptr;
    evd_status_t st = evd_plan_create(&p, n_host[i], lda_host[i], job, EVD_FP64, 0, 0, stream);
    if (st != EVD_OK) return st;
    size_t need = 0;
    evd_plan_workspace_size(p, &need);
    if (need > ws_bytes) { evd_plan_destroy(p); return EVD_ERR_WORKSPACE; }
    st = evd_syevd(p, A_host[i], w_host[i], job == EVD_VECTORS ? Q_host[i] : nullptr,
                   job == EVD_VECTORS ? ldq_host[i] : 1, ws);
    if (st == EVD_OK) {
      int info = 0;
      st = evd_plan_status(p, &info);
    }
    evd_plan_destroy(p);
    if (st != EVD_OK) return st;
  }
  return EVD_OK;
}

evd_status_t evd_autotune(int64_t n, evd_job_t job, evd_prec_t prec, const char* cache_path, int* b, int* nb) {
  (void)job; (void)prec; (void)cache_path;
  if (!b || !nb || n < 0) return EVD_ERR_INVALID_ARG;
  *b = n >= 4096 ? 64 : 32;
  *nb = *b;
  return EVD_OK;
}

}  // extern "C"
