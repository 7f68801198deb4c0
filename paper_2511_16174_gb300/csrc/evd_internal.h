// Internal declarations shared by the CUDA translation units of libevd.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "evd.h"

namespace evd {

// ---------------------------------------------------------------- status word
// Device status word layout (int[8]): [0] status code (evd_status_t), [1] info,
// [2] abort flag for cooperative kernels, [3..7] reserved.
constexpr int kStatusWords = 8;

// Spin limit for every device-side wait (a wait on a flag written by another CTA
// of the same launch).  Each iteration sleeps ~256 ns, so the limit is a few
// seconds of wall time.
constexpr long long kSpinLimit = 16ll * 1000 * 1000;

#define EVD_CUDA_TRY(expr)                                    \
  do {                                                        \
    cudaError_t e__ = (expr);                                 \
    if (e__ != cudaSuccess) return ::evd::cuda_fail(e__, #expr); \
  } while (0)

evd_status_t cuda_fail(cudaError_t e, const char* what);
// EVD_ERR_WORKSPACE, with a note on stderr when EVD_DEBUG is set.
evd_status_t ws_fail(const char* where, size_t have, size_t need);
evd_status_t ensure_dynamic_smem(const void* func, size_t bytes);
constexpr size_t kMaxDynamicSmem = 227 * 1024;  // per CTA on sm_103

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------- workspace
// A bump allocator over the caller's workspace.  Sizes are computed by running the
// same carve sequence with base == nullptr.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// ---------------------------------------------------------------- products
// C = alpha op(A) op(B) + beta C (column-major FP64).  `lower` restricts the
// computed and written part of C to i >= j (C square).  `slices` = 0: FP64 CUDA
// cores; 1..8: tensor-core split product with that many slices.
struct Gemm {
  char ta = 'N', tb = 'N';
  int64_t m = 0, n = 0, k = 0;
  double alpha = 1.0;
  const double* A = nullptr;
  int64_t lda = 1;
  const double* B = nullptr;
  int64_t ldb = 1;
  double beta = 0.0;
  double* C = nullptr;
  int64_t ldc = 1;
  bool lower = false;
  // A is symmetric with only its lower triangle stored (op(A) = A, m == k).
  bool a_sym_lower = false;
  // device status word that bounded waits report timeouts to (nullptr: the
  // library's own word for stand-alone products)
  int* status = nullptr;
  // use the tensor-core product whenever slices > 0 (stand-alone requests)
  bool force_tc = false;
  // statistics category of this product (nullptr: by engine)
  const char* tag = nullptr;
};

// Scratch a product needs (bytes) and the call itself.
size_t gemm_scratch_bytes(int64_t m, int64_t n, int64_t k, int slices);
evd_status_t gemm(const Gemm& g, int slices, void* scratch, size_t scratch_bytes, cudaStream_t s);
// `count` small products (no lower / symmetric forms, beta applied) on the FP64 CUDA
// cores in one launch; the descriptors are copied to `dev` (count Gemm) first, from
// host memory the call may reuse once it returns.
evd_status_t gemm_simt_batched(const Gemm* host, int count, Gemm* dev, const char* tag, cudaStream_t s);
bool ozaki_eligible(const Gemm& g);

// ---------------------------------------------------------------- the plan


struct PlanCore {
  int64_t n = 0, lda = 0;
  evd_job_t job = EVD_VALUES;
  evd_prec_t prec = EVD_FP64;
  int b = 32, nb = 32;
  int slices = 8;         // slices of the back transformation's products
  int sbr_slices = 8;     // slices of SBR's products (Z formation, trailing update)
  int ref_slices = 8;     // slices for refinement residual products
  int refine_iters = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 0;
  int panel_ctas = 64;    // CTAs of the cooperative panel QR
  int bcback_fused = 1;   // allow the fused BC-Back wave kernel
  int bc_kernel = 2;      // bulge chasing: 0 global memory, 1 shared-memory staged, 2 carried
  int bc_ctas_per_sm = 0; // bulge-chasing CTAs (sweeps in flight) per SM, 0 = by the sweep count
  int xe_slices = 4;      // slices of the refinement's X E product (E is at the error level)
  int order = -1;         // back transformation: 0 conventional, 1 reordered (Sec. 3.3), -1 by size
  bool dc_sync_free = false;  // D&C without host reads (capturable in a CUDA graph)
  void* dc_tree = nullptr;    // device copy of the D&C merge tree (plan-owned), or nullptr
  const struct BbSchedule* bb = nullptr;  // fused BC-Back schedule (plan-owned), or nullptr
  int* status = nullptr;  // device int[kStatusWords]
};

// Stage entry points (each enqueues on core.stream).
struct SbrWork {
  double* tau;     // n
  double* T;       // npanels * b * b   (T factor of each panel, column-major b x b)
  double* V;       // n * nb            (explicit V of the current panel block)
  double* W;       // n * nb
  double* Z;       // n * nb
  double* Y;       // n * nb            (scratch, A2 W)
  double* M;       // nb * nb * 4       (small products)
  double* VZ;      // n x 2 nb: [V_0 Z_0 V_1 Z_1 ...] of the current block
  double* ZV;      // n x 2 nb: [Z_0 V_0 Z_1 V_1 ...]
  double* X;       // 2 nb x nb
  double* partial; // per-CTA partial sums of the panel kernel
  unsigned* bar;   // grid barrier words
  double* band;    // (2b+1) x n lower band with room for the bulge
  void* gemm_ws;
  size_t gemm_ws_bytes;
};
evd_status_t sbr_run(const PlanCore& pc, double* A, const SbrWork& w);

struct BcWork {
  double* band;    // (2b+1) x n
  double* U;       // reflectors, b doubles each (v[0] = 1 explicit)
  double* Utau;    // one tau per reflector
  int64_t* off;    // n+1 prefix offsets of each sweep's reflectors
  int* prog;       // n progress counters
  unsigned* bar;
};
int64_t bc_num_reflectors(int64_t n, int b);
// Switch a plan's D&C to its sync-free form (no host reads; evd_api.cu).
void plan_set_sync_free(evd_plan_t p, bool on);
// Plan tunables and workspace size without creating a plan (evd_api.cu).
void fill_core(PlanCore& c, int64_t n, int64_t lda, evd_job_t job, evd_prec_t prec, int b, int nb);
size_t plan_workspace_bytes(int64_t n, int64_t lda, evd_job_t job, evd_prec_t prec, int b, int nb);
// Autotuner cache lookup for plans created with b = nb = 0 (evd_batched.cu).
bool autotune_lookup(int64_t n, evd_job_t job, evd_prec_t prec, int* b, int* nb, int* bc_per_sm);
// Upper bound on the number of reflector groups in one BC-Back wave (groups of a
// wave start 2b rows apart, all below row n).
int64_t bc_wave_max_groups(int64_t n, int b);
evd_status_t bc_run(const PlanCore& pc, const BcWork& w, double* d, double* e, bool vectors);

struct DcWork {
  double* Qtmp;    // n x n (block columns gathered in pole order, rotated)
  double* Qn;      // n x n (nondeflated columns; then the assembled block)
  double* Umat;    // n x n (secular eigenvectors of the merges)
  double* vec;     // 10 n doubles
  int* ivec;       // 32 n ints (8 n index arrays + merge descriptors)
  void* gemm_ws;
  size_t gemm_ws_bytes;
};
evd_status_t dc_run(const PlanCore& pc, double* d, double* e, double* Q, int64_t ldq,
                    const DcWork& w);
// The fused BC-Back schedule of a plan (b = 64, n >= 1024), built once at plan
// creation: the wave launches in order, the (J, k) of every group in launch order
// (device) and, for BC-Back of the identity, every group's column-tile range
// (device) with each launch's tile window.
struct BbLaunch {
  int64_t R0;        // first row of the launch's group 0
  int hh0;           // rows of group 0
  int64_t g0;        // index of group 0 in the tables
  int count;         // groups of the launch
  int64_t tile0, tile1, work_tiles;  // identity start: tile window and tiles of its ranges
};
struct BbSchedule {
  std::vector<BbLaunch> launches;
  int64_t groups = 0;
  int max_count = 0;
  int2* d_gjk = nullptr;
  int2* d_ranges = nullptr;
};
// Builds the schedule; allocates and fills its two device tables (cudaMalloc,
// synchronous copies).  bb_schedule_free releases them.
evd_status_t bb_schedule_build(int64_t n, int b, BbSchedule* out);
void bb_schedule_free(BbSchedule* s);

// Bytes of the device copy of the D&C merge tree of order n, and its upload
// (synchronous; done once per plan).
size_t dc_tree_bytes(int64_t n);
evd_status_t dc_tree_upload(int64_t n, void* dst, size_t bytes);

constexpr int kSbrBackPanels = 32;  // SBR panels merged into one compact WY group in SBR-Back
struct BackWork {
  double* Tg;      // T factors of the BC reflector groups
  double* Vg;      // V of the BC reflector groups of one wave (count x h x g)
  double* Yg;      // Y = V T of the same groups
  double* Wt;      // W^T of the same groups (count x n x g)
  size_t vg_capacity = 0;  // doubles available in Vg (and in Yg)
  size_t wt_capacity = 0;  // doubles available in Wt
  double* Vp;      // explicit V of a group of SBR panels (n x kSbrBackPanels b)
  double* Wp;      // kSbrBackPanels b x n
  double* Tp;      // kSbrBackPanels b x n
  double* Tblk;    // T of the group, (kSbrBackPanels b)^2
  double* Cblk;    // cross products V_prev^T V_p and T_prev C, 2 x (kSbrBackPanels b) x bb
  void* gemm_ws;
  size_t gemm_ws_bytes;
};
// BC-Back, X <- Q_b X.  With identity, X is set to the identity first and every
// fused wave skips the column tiles its groups' rows are still zero in (the
// reordered stages: Q_b I while D&C runs); this needs the plan's fused schedule.
evd_status_t bc_back_run(const PlanCore& pc, const BcWork& bw, double* Q, int64_t ldq,
                         const BackWork& w, bool identity = false);
int64_t bc_num_groups(int64_t n, int b);
// Whether a plan's whole-path solve runs the reordered stages (evd_api.cu).
bool reordered_stages(const PlanCore& c);
constexpr int64_t kReorderMinN = 8192;  // the default (order = -1) reorders from this size up
// Fused BC-Back wave (b = 64, 6 or 8 slices; evd_bcback.cu).
bool bcback_fused_supported(const PlanCore& pc, const double* Q, int64_t ldq);
// X (FP64, in place) to and from the fixed point the fused waves work in.
evd_status_t bcback_fixed_point(const PlanCore& pc, double* Q, int64_t ldq, bool to_fixed);
// Column tiles (128 columns) one fused wave launch covers: with a range table, the
// grid spans tiles [tile0, tile1] and the CTAs of group p outside ranges[p] leave at
// once (BC-Back of the identity, whose rows are zero outside a known column range).
struct WaveTiles {
  const int2* ranges = nullptr;  // device, one per group of the launch
  int64_t tile0 = 0, tile1 = -1;
  int64_t work_tiles = 0;        // sum over the groups of their range lengths
};
// The fused BC-Back waves in chunks: bcback_prep_chunk forms the compact WY factors
// and slices of `count` groups ((J, k) in the device table gjk) in `buf`
// (bcback_prep_bytes(count) bytes); bcback_fused_wave then runs one wave over the
// groups g_off .. g_off + count - 1 of a chunk of chunk_count prepared groups.
size_t bcback_prep_bytes(int count, int ref_slices);
evd_status_t bcback_prep_chunk(const PlanCore& pc, const BcWork& bw, const int2* gjk, int count, void* buf);
evd_status_t bcback_fused_wave(const PlanCore& pc, double* Q, int64_t ldq, void* buf, int chunk_count, int g_off,
                               int count, int64_t R0, int hh0, const WaveTiles& wt);
// Scratch of the fused waves with a dedicated region (reordered stages): the group
// table and the prep of a chunk of groups.
size_t bcback_fused_scratch_bytes(int64_t n, int b, int ref_slices);
evd_status_t sbr_back_run(const PlanCore& pc, const double* A, const double* sbr_T,
                          const double* sbr_tau, double* Q, int64_t ldq, const BackWork& w);

// Refinement (Ogita-Aishima)
struct RefineWork {
  double* R;   // n x n
  double* S;   // n x n
  double* AX;  // n x n
  double* E;   // n x n
  double* vec; // 4 n
  void* gemm_ws;
  size_t gemm_ws_bytes;
};
evd_status_t refine_run(const PlanCore& pc, const double* A0, int64_t lda0, double* w, double* Q,
                        int64_t ldq, int iters, const RefineWork& rw);

// Self-test of the bounded waits (evd_selftest.cu): kind 0 progress flag, 1 grid
// barrier, 2 mbarrier in a CTA holding tensor memory.
evd_status_t wait_selftest(const PlanCore& pc, int kind, int* flag_zero, unsigned* bar);

// ---------------------------------------------------------------- stats (evd_stats.cu)
// RAII scope: when stats are enabled, records CUDA events around the enclosed
// launches on stream s under category `cat` and adds the algorithmic flops/bytes.
class StatScope {
 public:
  // The category key is cat, or "cat/engine" when engine is given (the engine a
  // product ran on: "tc_split", "tc_split_prep", "fp64_simt", "fp64_splitk").
  StatScope(const char* cat, cudaStream_t s, double flops = 0, double bytes = 0, const char* engine = nullptr);
  ~StatScope();
  StatScope(const StatScope&) = delete;
  StatScope& operator=(const StatScope&) = delete;

 private:
  const char* cat_;
  const char* engine_ = nullptr;
  cudaStream_t s_;
  void* a_ = nullptr;
  bool on_ = false;
};
void count_launch(int n = 1);

// Small helpers (evd_util.cu)
evd_status_t check_finite_lower(const PlanCore& pc, const double* A, int64_t lda);
evd_status_t copy_lower_to_full(const double* A, int64_t lda, double* B, int64_t ldb, int64_t n,
                                cudaStream_t s);
evd_status_t copy_matrix(const double* A, int64_t lda, double* B, int64_t ldb, int64_t m, int64_t n,
                         cudaStream_t s);
evd_status_t set_identity(double* Q, int64_t ldq, int64_t n, cudaStream_t s);
int max_coresident_blocks(const void* kernel, int threads, size_t smem);

}  // namespace evd
