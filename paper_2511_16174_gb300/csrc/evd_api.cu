// C ABI of libevd: plans, workspace layout, the stage calls and the whole path.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "evd_internal.h"

using namespace evd;

namespace evd {
int64_t bc_num_reflectors(int64_t n, int b);
}

struct WsLayout {
  // persistent across the stages of one solve
  double* sbr_tau = nullptr;
  double* sbr_T = nullptr;
  double* band = nullptr;
  double* U = nullptr;
  double* Utau = nullptr;
  double* A0 = nullptr;     // split mode: copy of A for the refinement residuals
  double* Qd_int = nullptr; // values-only: D&C still forms Q_d here
  double* e = nullptr;      // sub-diagonal of T between BC and D&C
  // reordered stages only: Q_s Q_b (ld ldx), the scratch of the BC-Back waves while
  // D&C holds the union region and the product scratch, and the column-range table
  double* Xsb = nullptr;
  int64_t ldx = 0;
  char* bb_scratch = nullptr;
  size_t bb_bytes = 0;
  // union region
  char* uni = nullptr;
  size_t uni_bytes = 0;
  void* gemm_ws = nullptr;
  size_t gemm_bytes = 0;
  size_t total = 0;
};

struct evd_plan_s {
  PlanCore core;
  int* d_status = nullptr;   // kStatusWords ints
  unsigned* d_bar = nullptr; // 2 words
  int* d_prog = nullptr;     // n ints
  void* d_tree = nullptr;    // the D&C merge tree (uploaded once)
  BbSchedule* bb = nullptr;  // the fused BC-Back schedule (b = 64, n >= 1024, vectors)
  bool own_stream = false;
  // reordered stages: BC-Back of the identity on a high-priority stream and D&C on a
  // low-priority one, forked from and joined back to the plan's stream with events
  cudaStream_t hi = nullptr, lo = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join_hi = nullptr, ev_join_lo = nullptr;
};

namespace {

int64_t n_panels(int64_t n, int b) {
  int64_t np = 0;
  while (n - (np * b + b) >= 2) ++np;
  return np;
}

constexpr int kMaxPanelCtas = 2048;

size_t sbr_union_bytes(int64_t n, int b, int nb) {
  Carver c(nullptr);
  c.take<double>((size_t)n * b);  // V
  c.take<double>((size_t)n * b);  // W
  c.take<double>((size_t)n * b);  // Z
  c.take<double>((size_t)n * b);  // Y
  c.take<double>((size_t)b * b * 4);
  c.take<double>((size_t)2 * kMaxPanelCtas * (2 + b) + (size_t)b * b);
  c.take<double>((size_t)n * 2 * nb);  // VZ
  c.take<double>((size_t)n * 2 * nb);  // ZV
  c.take<double>((size_t)2 * nb * nb); // X
  return c.off;
}
size_t dc_union_bytes(int64_t n) {
  Carver c(nullptr);
  c.take<double>((size_t)n * n);
  c.take<double>((size_t)n * n);
  c.take<double>((size_t)n * n);
  c.take<double>((size_t)10 * n + 8);
  c.take<int>((size_t)32 * n + 1024);
  return c.off;
}
size_t back_union_bytes(int64_t n, int b) {
  Carver c(nullptr);
  const int64_t K = (int64_t)kSbrBackPanels * b;
  c.take<double>((size_t)n * K);
  c.take<double>((size_t)n * K);
  c.take<double>((size_t)n * K);
  c.take<double>((size_t)K * K);
  c.take<double>((size_t)2 * K * b);
  const int64_t pmax = bc_wave_max_groups(n, b), h = 2 * b - 1;
  c.take<double>((size_t)pmax * h * b);
  c.take<double>((size_t)pmax * h * b);
  c.take<double>((size_t)pmax * n * b);
  return c.off;
}
size_t refine_union_bytes(int64_t n) {
  Carver c(nullptr);
  c.take<double>((size_t)n * n);
  c.take<double>((size_t)n * n);
  c.take<double>((size_t)n * n);
  c.take<double>((size_t)4 * n + 8);
  return c.off;
}

WsLayout make_layout(const PlanCore& pc, void* ws) {
  WsLayout L;
  const int64_t n = pc.n;
  const int b = pc.b;
  Carver c(ws);
  L.sbr_tau = c.take<double>((size_t)std::max<int64_t>(n, 1));
  L.sbr_T = c.take<double>((size_t)std::max<int64_t>(n_panels(n, b), 1) * b * b);
  L.band = c.take<double>((size_t)(2 * b + 1) * std::max<int64_t>(n, 1));
  L.e = c.take<double>((size_t)std::max<int64_t>(n, 1));
  if (pc.job == EVD_VECTORS) {
    int64_t nref = bc_num_reflectors(n, b);
    L.U = c.take<double>((size_t)std::max<int64_t>(nref, 1) * b);
    L.Utau = c.take<double>((size_t)std::max<int64_t>(nref, 1));
  } else {
    L.Qd_int = c.take<double>((size_t)n * n);
  }
  if (pc.prec == EVD_SPLIT_BF16) L.A0 = c.take<double>((size_t)n * n);
  if (reordered_stages(pc)) {
    L.ldx = n + (n & 1);  // even: the fused waves' tensor copies want a 16-byte column stride
    L.Xsb = c.take<double>((size_t)L.ldx * n);
    L.bb_bytes = bcback_fused_scratch_bytes(n, b, pc.ref_slices);
    L.bb_scratch = c.take<char>(L.bb_bytes);
  }
  size_t ub = std::max({sbr_union_bytes(n, b, pc.nb), dc_union_bytes(n), back_union_bytes(n, b),
                        pc.prec == EVD_SPLIT_BF16 ? refine_union_bytes(n) : (size_t)0});
  L.uni = c.take<char>(ub);
  L.uni_bytes = ub;
  // the D&C merges and the refinement residuals run at ref_slices in every mode
  size_t gb = std::max({gemm_scratch_bytes(n, n, n, pc.slices), gemm_scratch_bytes(n, n, n, pc.ref_slices),
                        gemm_scratch_bytes(n, n, n, pc.sbr_slices)});
  L.gemm_ws = c.take<char>(gb);
  L.gemm_bytes = gb;
  L.total = align_up(c.off, 256);
  return L;
}

SbrWork sbr_work(const evd_plan_s* p, const WsLayout& L) {
  const int64_t n = p->core.n;
  const int b = p->core.b;
  Carver c(L.uni);
  SbrWork w;
  w.tau = L.sbr_tau;
  w.T = L.sbr_T;
  w.V = c.take<double>((size_t)n * b);
  w.W = c.take<double>((size_t)n * b);
  w.Z = c.take<double>((size_t)n * b);
  w.Y = c.take<double>((size_t)n * b);
  w.M = c.take<double>((size_t)b * b * 4);
  w.partial = c.take<double>((size_t)2 * kMaxPanelCtas * (2 + b) + (size_t)b * b);
  w.VZ = c.take<double>((size_t)n * 2 * p->core.nb);
  w.ZV = c.take<double>((size_t)n * 2 * p->core.nb);
  w.X = c.take<double>((size_t)2 * p->core.nb * p->core.nb);
  w.bar = p->d_bar;
  w.band = L.band;
  w.gemm_ws = L.gemm_ws;
  w.gemm_ws_bytes = L.gemm_bytes;
  return w;
}

BcWork bc_work(const evd_plan_s* p, const WsLayout& L) {
  BcWork w;
  w.band = L.band;
  w.U = L.U;
  w.Utau = L.Utau;
  w.off = nullptr;
  w.prog = p->d_prog;
  w.bar = p->d_bar;
  return w;
}

DcWork dc_work(const evd_plan_s* p, const WsLayout& L) {
  const int64_t n = p->core.n;
  Carver c(L.uni);
  DcWork w;
  w.Qtmp = c.take<double>((size_t)n * n);
  w.Qn = c.take<double>((size_t)n * n);
  w.Umat = c.take<double>((size_t)n * n);
  w.vec = c.take<double>((size_t)10 * n + 8);
  w.ivec = c.take<int>((size_t)32 * n + 1024);
  w.gemm_ws = L.gemm_ws;
  w.gemm_ws_bytes = L.gemm_bytes;
  return w;
}

BackWork back_work(const evd_plan_s* p, const WsLayout& L) {
  const int64_t n = p->core.n;
  const int b = p->core.b;
  Carver c(L.uni);
  BackWork w;
  w.Tg = nullptr;
  const int64_t K = (int64_t)kSbrBackPanels * b;
  w.Vp = c.take<double>((size_t)n * K);
  w.Wp = c.take<double>((size_t)n * K);
  w.Tp = c.take<double>((size_t)n * K);
  w.Tblk = c.take<double>((size_t)K * K);
  w.Cblk = c.take<double>((size_t)2 * K * b);
  const int64_t pmax = bc_wave_max_groups(n, b), h = 2 * b - 1;
  w.Vg = c.take<double>((size_t)pmax * h * b);
  w.Yg = c.take<double>((size_t)pmax * h * b);
  w.Wt = c.take<double>((size_t)pmax * n * b);
  w.vg_capacity = (size_t)pmax * h * b;
  w.wt_capacity = (size_t)pmax * n * b;
  w.gemm_ws = L.gemm_ws;
  w.gemm_ws_bytes = L.gemm_bytes;
  return w;
}

RefineWork refine_work(const evd_plan_s* p, const WsLayout& L) {
  const int64_t n = p->core.n;
  Carver c(L.uni);
  RefineWork w;
  w.R = c.take<double>((size_t)n * n);
  w.S = c.take<double>((size_t)n * n);
  w.AX = c.take<double>((size_t)n * n);
  w.E = nullptr;
  w.vec = c.take<double>((size_t)4 * n + 8);
  w.gemm_ws = L.gemm_ws;
  w.gemm_ws_bytes = L.gemm_bytes;
  return w;
}

evd_status_t check_ws(const evd_plan_s* p, void* ws) {
  if (!ws && p->core.n > 0) return EVD_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return EVD_ERR_WORKSPACE;
  return EVD_OK;
}

int default_b(int64_t n) { return n >= 4096 ? 64 : 32; }

}  // namespace

namespace evd {

// Reordered stages (Sec. 3.3): the back transformation is applied to the identity,
// Q_sb = Q_s Q_b, while D&C computes Q_d on a side stream, and Q = Q_sb Q_d is one
// more product.  It needs the fused BC-Back waves (b = 64, 6 or 8 slices).
bool reordered_stages(const PlanCore& c) {
  const bool eligible = c.job == EVD_VECTORS && c.b == 64 && (c.slices == 6 || c.slices == 8) && c.n >= 1024 &&
                        c.n < ((int64_t)1 << 31) && c.bcback_fused;
  if (c.order == 0) return false;
  if (c.order == 1) return eligible;
  return eligible && c.n >= kReorderMinN;
}

// The plan's tunables.  b = nb = 0: the autotuner's cached choice (file named by
// EVD_AUTOTUNE_CACHE) if there is one, else b = 64 for n >= 4096 and 32 below,
// nb = 16 b for n >= 32768, 8 b for n >= 16384 and b below.  b > 0, nb = 0: nb = b.
void fill_core(PlanCore& c, int64_t n, int64_t lda, evd_job_t job, evd_prec_t prec, int b, int nb) {
  c.n = n;
  c.lda = lda;
  c.job = job;
  c.prec = prec;
  int tb = 0, tnb = 0, tper = 0;
  if (b == 0 && nb == 0 && autotune_lookup(n, job, prec, &tb, &tnb, &tper)) {
    c.b = tb;
    c.nb = tnb;
    c.bc_ctas_per_sm = tper;
  } else {
    c.b = (b > 0) ? b : default_b(n);
    if (c.b < 2 && b == 0) c.b = 2;
    // double blocking pays once the trailing matrix is large (fewer, wider syr2k,
    // one split of the stale trailing matrix per block)
    const int dbl = (b != 0) ? 1 : (n >= 32768) ? 16 : (n >= 16384) ? 8 : 1;
    c.nb = (nb > 0) ? nb : dbl * c.b;
  }
  // split precision: 6 slices (21 slice pairs instead of 36) leave the eigenvectors
  // accurate enough (about 1e-11 at n ~ 1e3) for two refinement steps to resolve
  // clusters of gap 1e-6; with 4 slices (about 1e-7) such clusters stay mixed.
  c.slices = (prec == EVD_SPLIT_BF16) ? 6 : 8;
  // the reduction's product error is a backward error of A: it leaves a coupling
  // between nearly equal eigenvalues that the refinement keeps (a pair inside its
  // threshold is not rotated), so SBR keeps 7 slices (2^-48) in split mode; errors of
  // the back transformation only perturb X and are refined away
  c.sbr_slices = (prec == EVD_SPLIT_BF16) ? 7 : 8;
  c.ref_slices = 8;
  c.refine_iters = (prec == EVD_SPLIT_BF16) ? 2 : 0;
}

size_t plan_workspace_bytes(int64_t n, int64_t lda, evd_job_t job, evd_prec_t prec, int b, int nb) {
  PlanCore c;
  fill_core(c, n, lda, job, prec, b, nb);
  return make_layout(c, nullptr).total;
}

}  // namespace evd

extern "C" {

const char* evd_status_string(evd_status_t s) {
  switch (s) {
    case EVD_OK: return "EVD_OK";
    case EVD_ERR_INVALID_ARG: return "EVD_ERR_INVALID_ARG";
    case EVD_ERR_WORKSPACE: return "EVD_ERR_WORKSPACE";
    case EVD_ERR_OOM: return "EVD_ERR_OOM";
    case EVD_ERR_CUDA: return "EVD_ERR_CUDA";
    case EVD_ERR_NONFINITE: return "EVD_ERR_NONFINITE";
    case EVD_ERR_NO_CONVERGENCE: return "EVD_ERR_NO_CONVERGENCE";
    case EVD_ERR_TIMEOUT: return "EVD_ERR_TIMEOUT";
    case EVD_ERR_NOT_SUPPORTED: return "EVD_ERR_NOT_SUPPORTED";
  }
  return "EVD_ERR_UNKNOWN";
}

evd_status_t evd_plan_create(evd_plan_t* plan, int64_t n, int64_t lda, evd_job_t job, evd_prec_t prec, int b, int nb,
                             void* stream) {
  if (!plan) return EVD_ERR_INVALID_ARG;
  *plan = nullptr;
  if (n < 0 || lda < std::max<int64_t>(1, n) || b < 0 || nb < 0 || b > 128) return EVD_ERR_INVALID_ARG;
  if (b > 0 && nb > 0 && nb % b != 0) return EVD_ERR_INVALID_ARG;
  if (job != EVD_VALUES && job != EVD_VECTORS) return EVD_ERR_INVALID_ARG;
  if (prec == EVD_SPLIT_INT8) return EVD_ERR_NOT_SUPPORTED;
  if (prec != EVD_FP64 && prec != EVD_SPLIT_BF16) return EVD_ERR_INVALID_ARG;
  if (n >= (int64_t)1 << 31) return EVD_ERR_INVALID_ARG;
  if (prec == EVD_SPLIT_BF16 && job != EVD_VECTORS) return EVD_ERR_INVALID_ARG;
  evd_plan_s* p = new (std::nothrow) evd_plan_s();
  if (!p) return EVD_ERR_OOM;
  PlanCore& c = p->core;
  fill_core(c, n, lda, job, prec, b, nb);
  c.stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&c.device);
  cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, c.device);
  const size_t tree_bytes = dc_tree_bytes(n);
  if (cudaMalloc(&p->d_status, sizeof(int) * kStatusWords) != cudaSuccess ||
      cudaMalloc(&p->d_bar, sizeof(unsigned) * 4) != cudaSuccess ||
      cudaMalloc(&p->d_prog, sizeof(int) * std::max<int64_t>(n, 1)) != cudaSuccess ||
      cudaMalloc(&p->d_tree, tree_bytes) != cudaSuccess) {
    cudaFree(p->d_status);
    cudaFree(p->d_bar);
    cudaFree(p->d_prog);
    cudaFree(p->d_tree);
    (void)cudaGetLastError();
    delete p;
    return EVD_ERR_OOM;
  }
  if (dc_tree_upload(n, p->d_tree, tree_bytes) != EVD_OK) {
    evd_plan_destroy(p);
    return EVD_ERR_CUDA;
  }
  c.dc_tree = p->d_tree;
  if (job == EVD_VECTORS && c.b == 64 && n >= 1024) {
    p->bb = new (std::nothrow) BbSchedule();
    if (!p->bb) {
      evd_plan_destroy(p);
      return EVD_ERR_OOM;
    }
    const evd_status_t bst = bb_schedule_build(n, c.b, p->bb);
    if (bst != EVD_OK) {
      evd_plan_destroy(p);
      return bst;
    }
    c.bb = p->bb;
  }
  cudaMemset(p->d_status, 0, sizeof(int) * kStatusWords);
  cudaMemset(p->d_bar, 0, sizeof(unsigned) * 4);
  c.status = p->d_status;
  *plan = p;
  return EVD_OK;
}

evd_status_t evd_plan_set_option(evd_plan_t p, evd_option_t opt, int value) {
  if (!p) return EVD_ERR_INVALID_ARG;
  PlanCore& c = p->core;
  switch (opt) {
    case EVD_OPT_SLICES:
      if (value < 1 || value > 8) return EVD_ERR_INVALID_ARG;
      c.slices = value;
      return EVD_OK;
    case EVD_OPT_SBR_SLICES:
      if (value < 1 || value > 8) return EVD_ERR_INVALID_ARG;
      c.sbr_slices = value;
      return EVD_OK;
    case EVD_OPT_REFINE_ITERS:
      if (value < 0 || value > 8) return EVD_ERR_INVALID_ARG;
      c.refine_iters = value;
      return EVD_OK;
    case EVD_OPT_BCBACK_FUSED:
      if (value != 0 && value != 1) return EVD_ERR_INVALID_ARG;
      c.bcback_fused = value;
      return EVD_OK;
    case EVD_OPT_BC_KERNEL:
      if (value < 0 || value > 2) return EVD_ERR_INVALID_ARG;
      c.bc_kernel = value;
      return EVD_OK;
    case EVD_OPT_PANEL_CTAS:
      if (value < 1 || value > kMaxPanelCtas) return EVD_ERR_INVALID_ARG;
      c.panel_ctas = value;
      return EVD_OK;
    case EVD_OPT_XE_SLICES:
      if (value < 1 || value > 8) return EVD_ERR_INVALID_ARG;
      c.xe_slices = value;
      return EVD_OK;
    case EVD_OPT_BC_CTAS_PER_SM:
      if (value < 0 || value > 4) return EVD_ERR_INVALID_ARG;
      c.bc_ctas_per_sm = value;
      return EVD_OK;
    case EVD_OPT_ORDER:
      if (value < -1 || value > 1) return EVD_ERR_INVALID_ARG;
      c.order = value;
      return EVD_OK;
  }
  return EVD_ERR_INVALID_ARG;
}

evd_status_t evd_plan_get_option(evd_plan_t p, evd_option_t opt, int* value) {
  if (!p || !value) return EVD_ERR_INVALID_ARG;
  const PlanCore& c = p->core;
  switch (opt) {
    case EVD_OPT_SLICES: *value = c.slices; return EVD_OK;
    case EVD_OPT_SBR_SLICES: *value = c.sbr_slices; return EVD_OK;
    case EVD_OPT_REFINE_ITERS: *value = c.refine_iters; return EVD_OK;
    case EVD_OPT_BCBACK_FUSED: *value = c.bcback_fused; return EVD_OK;
    case EVD_OPT_BC_KERNEL: *value = c.bc_kernel; return EVD_OK;
    case EVD_OPT_PANEL_CTAS: *value = c.panel_ctas; return EVD_OK;
    case EVD_OPT_XE_SLICES: *value = c.xe_slices; return EVD_OK;
    case EVD_OPT_BC_CTAS_PER_SM: *value = c.bc_ctas_per_sm; return EVD_OK;
    case EVD_OPT_ORDER: *value = reordered_stages(c) ? 1 : 0; return EVD_OK;
  }
  return EVD_ERR_INVALID_ARG;
}

}  // extern "C"

namespace evd {
void plan_set_sync_free(evd_plan_t p, bool on) {
  if (p) p->core.dc_sync_free = on;
}
}  // namespace evd

extern "C" {

evd_status_t evd_wait_selftest(evd_plan_t p, int kind) {
  if (!p || kind < 0 || kind > 2) return EVD_ERR_INVALID_ARG;
  return wait_selftest(p->core, kind, p->d_prog, p->d_bar);
}

evd_status_t evd_plan_get_blocking(evd_plan_t p, int* b, int* nb) {
  if (!p) return EVD_ERR_INVALID_ARG;
  if (b) *b = p->core.b;
  if (nb) *nb = p->core.nb;
  return EVD_OK;
}

evd_status_t evd_plan_workspace_size(evd_plan_t p, size_t* bytes) {
  if (!p || !bytes) return EVD_ERR_INVALID_ARG;
  *bytes = make_layout(p->core, nullptr).total;
  return EVD_OK;
}

evd_status_t evd_sbr(evd_plan_t p, double* A, void* ws) {
  if (!p || (!A && p->core.n > 0)) return EVD_ERR_INVALID_ARG;
  evd_status_t st = check_ws(p, ws);
  if (st != EVD_OK) return st;
  if (p->core.n == 0) return EVD_OK;
  WsLayout L = make_layout(p->core, ws);
  st = check_finite_lower(p->core, A, p->core.lda);
  if (st != EVD_OK) return st;
  return sbr_run(p->core, A, sbr_work(p, L));
}

evd_status_t evd_bulge_chase(evd_plan_t p, void* ws, double* d, double* e) {
  if (!p || ((!d || (!e && p->core.n > 1)) && p->core.n > 0)) return EVD_ERR_INVALID_ARG;
  evd_status_t st = check_ws(p, ws);
  if (st != EVD_OK) return st;
  if (p->core.n == 0) return EVD_OK;
  WsLayout L = make_layout(p->core, ws);
  return bc_run(p->core, bc_work(p, L), d, e, p->core.job == EVD_VECTORS);
}

evd_status_t evd_tridiag_solve(evd_plan_t p, double* d, double* e, double* Qd, int64_t ldq, void* ws) {
  if (!p || (p->core.n > 0 && !d)) return EVD_ERR_INVALID_ARG;
  evd_status_t st = check_ws(p, ws);
  if (st != EVD_OK) return st;
  const int64_t n = p->core.n;
  if (n == 0) return EVD_OK;
  if (n > 1 && !e) return EVD_ERR_INVALID_ARG;
  WsLayout L = make_layout(p->core, ws);
  double* Q = Qd;
  int64_t ld = ldq;
  if (!Q) {
    if (!L.Qd_int) return EVD_ERR_INVALID_ARG;  // a vectors plan must be given Qd
    Q = L.Qd_int;
    ld = n;
  } else if (ldq < n) {
    return EVD_ERR_INVALID_ARG;
  }
  return dc_run(p->core, d, e, Q, ld, dc_work(p, L));
}

evd_status_t evd_back_transform(evd_plan_t p, const double* A_reduced, void* ws, double* Q, int64_t ldq) {
  if (!p || p->core.job != EVD_VECTORS) return EVD_ERR_INVALID_ARG;
  const int64_t n = p->core.n;
  if (n == 0) return EVD_OK;
  if (!A_reduced || !Q || ldq < n) return EVD_ERR_INVALID_ARG;
  evd_status_t st = check_ws(p, ws);
  if (st != EVD_OK) return st;
  WsLayout L = make_layout(p->core, ws);
  BackWork bw = back_work(p, L);
  st = bc_back_run(p->core, bc_work(p, L), Q, ldq, bw);
  if (st != EVD_OK) return st;
  return sbr_back_run(p->core, A_reduced, L.sbr_T, L.sbr_tau, Q, ldq, bw);
}

evd_status_t evd_refine(evd_plan_t p, const double* A0, double* w, double* Q, int64_t ldq, int iterations, void* ws) {
  if (!p || p->core.prec != EVD_SPLIT_BF16) return EVD_ERR_INVALID_ARG;
  const int64_t n = p->core.n;
  if (n == 0) return EVD_OK;
  if (!A0 || !w || !Q || ldq < n || iterations < 0) return EVD_ERR_INVALID_ARG;
  evd_status_t st = check_ws(p, ws);
  if (st != EVD_OK) return st;
  WsLayout L = make_layout(p->core, ws);
  return refine_run(p->core, A0, p->core.lda, w, Q, ldq, iterations, refine_work(p, L));
}

namespace {

evd_status_t ensure_side_streams(evd_plan_t p) {
  if (p->hi) return EVD_OK;
  int least = 0, greatest = 0;
  EVD_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  EVD_CUDA_TRY(cudaStreamCreateWithPriority(&p->hi, cudaStreamNonBlocking, greatest));
  EVD_CUDA_TRY(cudaStreamCreateWithPriority(&p->lo, cudaStreamNonBlocking, least));
  EVD_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
  EVD_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_join_hi, cudaEventDisableTiming));
  EVD_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_join_lo, cudaEventDisableTiming));
  return EVD_OK;
}

// Stages 3 and 4 in the reordered order (Sec. 3.3).  On entry (d, e) = (w, etmp) hold
// T and ws the BC and SBR reflectors.  D&C runs on the plan's low-priority stream,
// issued from a host thread of its own (its merges read deflation counts on the
// host), and writes Q_d into Q.  Meanwhile the high-priority stream computes
// X = Q_b I in ws (the fused waves skip the column tiles that are still zero): its
// CTAs are dispatched first, and D&C's small FP64 kernels run in the room a wave CTA
// leaves on its SM.  Once both are done (D&C holds the union region and the product
// scratch), the plan's stream applies X <- Q_s X and forms Q = X Q_d.
evd_status_t reordered_back(evd_plan_t p, const WsLayout& L, const double* A, double* w, double* etmp, double* Q,
                            int64_t ldq) {
  const PlanCore& pc = p->core;
  cudaStream_t s0 = pc.stream;
  evd_status_t st = ensure_side_streams(p);
  if (st != EVD_OK) return st;
  EVD_CUDA_TRY(cudaEventRecord(p->ev_fork, s0));
  EVD_CUDA_TRY(cudaStreamWaitEvent(p->hi, p->ev_fork, 0));
  EVD_CUDA_TRY(cudaStreamWaitEvent(p->lo, p->ev_fork, 0));
  PlanCore cs = pc;
  cs.stream = p->lo;
  PlanCore ch = pc;
  ch.stream = p->hi;
  const DcWork dw = dc_work(p, L);
  evd_status_t st_dc = EVD_OK;
  std::thread dc_thread([&] {
    if (cudaSetDevice(pc.device) != cudaSuccess) {
      st_dc = EVD_ERR_CUDA;
      return;
    }
    st_dc = dc_run(cs, w, etmp, Q, ldq, dw);
  });
  BackWork bw;
  bw.gemm_ws = L.bb_scratch;
  bw.gemm_ws_bytes = L.bb_bytes;
  st = bc_back_run(ch, bc_work(p, L), L.Xsb, L.ldx, bw, true);
  dc_thread.join();
  // join whatever both streams queued, even after an error, so that the order holds
  cudaEventRecord(p->ev_join_hi, p->hi);
  cudaEventRecord(p->ev_join_lo, p->lo);
  cudaStreamWaitEvent(s0, p->ev_join_hi, 0);
  cudaStreamWaitEvent(s0, p->ev_join_lo, 0);
  if (st != EVD_OK) return st;
  if (st_dc != EVD_OK) return st_dc;
  st = sbr_back_run(pc, A, L.sbr_T, L.sbr_tau, L.Xsb, L.ldx, back_work(p, L));
  if (st != EVD_OK) return st;
  // Q = X Q_d.  C is B: the split product reads B only while splitting it into the
  // scratch, before the tensor-core kernel writes C (beta = 0).
  Gemm gf;
  gf.m = pc.n; gf.n = pc.n; gf.k = pc.n; gf.A = L.Xsb; gf.lda = L.ldx; gf.B = Q; gf.ldb = ldq;
  gf.C = Q; gf.ldc = ldq; gf.alpha = 1.0; gf.beta = 0.0;
  gf.force_tc = true; gf.status = pc.status; gf.tag = "final_gemm";
  return gemm(gf, pc.slices, L.gemm_ws, L.gemm_bytes, s0);
}

}  // namespace

evd_status_t evd_syevd(evd_plan_t p, double* A, double* w, double* Q, int64_t ldq, void* ws) {
  if (!p) return EVD_ERR_INVALID_ARG;
  const int64_t n = p->core.n;
  if (n == 0) return EVD_OK;
  if (!A || !w) return EVD_ERR_INVALID_ARG;
  const bool vec = p->core.job == EVD_VECTORS;
  if (vec && (!Q || ldq < n)) return EVD_ERR_INVALID_ARG;
  evd_status_t st = check_ws(p, ws);
  if (st != EVD_OK) return st;
  WsLayout L = make_layout(p->core, ws);
  if (p->core.prec == EVD_SPLIT_BF16) {
    st = copy_matrix(A, p->core.lda, L.A0, n, n, n, p->core.stream);
    if (st != EVD_OK) return st;
  }
  st = evd_sbr(p, A, ws);
  if (st != EVD_OK) return st;
  double* etmp = L.e;
  st = evd_bulge_chase(p, ws, w, etmp);
  if (st != EVD_OK) return st;
  if (!(vec && reordered_stages(p->core))) {
    st = evd_tridiag_solve(p, w, etmp, vec ? Q : nullptr, ldq, ws);
    if (st != EVD_OK) return st;
  }
  if (!vec) return EVD_OK;
  st = reordered_stages(p->core) ? reordered_back(p, L, A, w, etmp, Q, ldq) : evd_back_transform(p, A, ws, Q, ldq);
  if (st != EVD_OK) return st;
  if (p->core.prec == EVD_SPLIT_BF16 && p->core.refine_iters > 0)
    st = refine_run(p->core, L.A0, n, w, Q, ldq, p->core.refine_iters, refine_work(p, L));
  return st;
}

evd_status_t evd_plan_status(evd_plan_t p, int* info) {
  if (!p) return EVD_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(p->core.stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return EVD_ERR_CUDA;
  }
  int h[kStatusWords] = {0};
  if (cudaMemcpy(h, p->d_status, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return EVD_ERR_CUDA;
  cudaMemset(p->d_status, 0, sizeof(int) * kStatusWords);
  // a grid barrier that gave up leaves its arrival count behind
  if (h[0] != 0 || h[2] != 0) cudaMemset(p->d_bar, 0, sizeof(unsigned) * 4);
  if (info) *info = h[1];
  return static_cast<evd_status_t>(h[0]);
}

void evd_plan_destroy(evd_plan_t p) {
  if (!p) return;
  cudaStreamSynchronize(p->core.stream);
  if (p->hi) {
    cudaStreamSynchronize(p->hi);
    cudaStreamSynchronize(p->lo);
    cudaStreamDestroy(p->hi);
    cudaStreamDestroy(p->lo);
    cudaEventDestroy(p->ev_fork);
    cudaEventDestroy(p->ev_join_hi);
    cudaEventDestroy(p->ev_join_lo);
  }
  cudaFree(p->d_status);
  cudaFree(p->d_bar);
  cudaFree(p->d_prog);
  cudaFree(p->d_tree);
  if (p->bb) {
    bb_schedule_free(p->bb);
    delete p->bb;
  }
  delete p;
}

// ---------------------------------------------------------------- product engine
evd_status_t evd_gemm_workspace_size(int64_t m, int64_t n, int64_t k, int slices, size_t* bytes) {
  if (!bytes || m < 0 || n < 0 || k < 0 || slices < 0 || slices > 8) return EVD_ERR_INVALID_ARG;
  *bytes = gemm_scratch_bytes(m, n, k, slices);
  return EVD_OK;
}

evd_status_t evd_dgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                       int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int slices,
                       void* ws, size_t ws_bytes, void* stream) {
  transa = (char)toupper(transa);
  transb = (char)toupper(transb);
  if ((transa != 'N' && transa != 'T') || (transb != 'N' && transb != 'T')) return EVD_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0 || slices < 0 || slices > 8) return EVD_ERR_INVALID_ARG;
  const int64_t ar = (transa == 'N') ? m : k, br = (transb == 'N') ? k : n;
  if (lda < std::max<int64_t>(1, ar) || ldb < std::max<int64_t>(1, br) || ldc < std::max<int64_t>(1, m))
    return EVD_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && (!C || (k > 0 && (!A || !B)))) return EVD_ERR_INVALID_ARG;
  if (ws_bytes < gemm_scratch_bytes(m, n, k, slices)) return EVD_ERR_WORKSPACE;
  Gemm g;
  g.ta = transa; g.tb = transb; g.m = m; g.n = n; g.k = k; g.alpha = alpha; g.A = A; g.lda = lda;
  g.B = B; g.ldb = ldb; g.beta = beta; g.C = C; g.ldc = ldc;
  g.force_tc = true;
  return gemm(g, slices, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
