/*
 * evd.h -- C ABI of libevd, a GB300 (sm_103a) two-stage symmetric eigensolver.
 *
 * Problem (Sec. 1): for a dense symmetric A (n x n), compute A = Q Lambda Q^T with
 * Lambda = diag(w) ascending and Q orthogonal.  The method is the two-stage EVD of
 * Sec. 2.1: successive band reduction (SBR, Sec. 2.1.1 and Eq. 1) to a band of
 * half-width b, bulge chasing (BC, Sec. 2.1.1 and Sec. 4.2) to a tridiagonal T, a
 * divide-and-conquer tridiagonal solve (Sec. 1, Sec. 3.3), and the back
 * transformation (Sec. 2.1.2: BC-Back then SBR-Back, conventional order).
 *
 * Conventions for every entry point:
 *   - Matrices are FP64, column-major: element (i, j) at ptr[i + j*ld], ld >= n.
 *   - Only the LOWER triangle of A is read (Sec. 4.1 keeps the lower triangle).
 *   - All matrix and vector pointers are DEVICE pointers unless the argument
 *     name ends in _host.  The caller owns every buffer (A, w, d, e, Q and the
 *     workspace); the library never frees them.  A plan owns only small internal
 *     state (status word, progress counters, tuning choices).
 *   - Calls are asynchronous on the plan's stream.  Errors that the host can see
 *     (bad sizes, null pointers, too small a workspace) return at once.  Errors
 *     found on the device (non-finite input, a wait that timed out,
 *     non-convergence) are latched in the plan's status word and returned by
 *     evd_plan_status().  No call ever falls back to the CPU.
 *   - No C++ exception crosses this ABI.
 */
#ifndef EVD_H_
#define EVD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct evd_plan_s* evd_plan_t;

typedef enum {
  EVD_OK = 0,
  EVD_ERR_INVALID_ARG = 1,     /* a size, leading dimension or pointer is invalid        */
  EVD_ERR_WORKSPACE = 2,       /* workspace pointer null or smaller than required        */
  EVD_ERR_OOM = 3,             /* the plan's small internal allocation failed            */
  EVD_ERR_CUDA = 4,            /* a CUDA runtime call failed                             */
  EVD_ERR_NONFINITE = 5,       /* the input held NaN or Inf (device check)               */
  EVD_ERR_NO_CONVERGENCE = 6,  /* a tridiagonal leaf or secular root did not converge    */
  EVD_ERR_TIMEOUT = 7,         /* a bounded device-side wait gave up                     */
  EVD_ERR_NOT_SUPPORTED = 8    /* option not built for this GPU                          */
} evd_status_t;

typedef enum { EVD_VALUES = 0, EVD_VECTORS = 1 } evd_job_t;

/* Arithmetic of the dense contractions (the SBR trailing update and Z formation
 * of Eq. 1, the back-transformation GEMMs and the divide-and-conquer merges).
 *   EVD_FP64        FP64-accurate products: FP64 operands split into 8 bfloat16
 *                   slices of 7 bits, slice pairs multiplied on tensor cores with
 *                   exact FP32 partial sums, recombined in 64-bit integers.  The
 *                   fused BC-Back waves (b = 64) use 7 float16 digits of 8 bits
 *                   (55 bits) with the same exact accumulation.
 *   EVD_SPLIT_BF16  Split precision: 7 slices for SBR's products, 6 for SBR-Back
 *                   and the final product (the fused BC-Back waves keep their 7
 *                   digits), then Ogita-Aishima refinement with FP64-accurate
 *                   residual products (D&C merges stay FP64-accurate).
 *   EVD_SPLIT_INT8  Accepted for interface completeness; GB300's INT8 tensor rate
 *                   is far below its BF16 rate, so this returns EVD_ERR_NOT_SUPPORTED.
 * Householder vectors and tau (panel QR, BC), the secular equation and the
 * refinement residual products are FP64-accurate in every mode. */
typedef enum { EVD_FP64 = 0, EVD_SPLIT_INT8 = 1, EVD_SPLIT_BF16 = 2 } evd_prec_t;

/* Create a plan for n x n problems with leading dimension lda.
 *   b   band half-width of SBR (Sec. 2.1.1; typical 32, Sec. 4.1).
 *   nb  outer (double-blocking) width of SBR, a multiple of b.
 *   b = nb = 0: the autotuner's cached choice (see evd_autotune), else b = 64 for
 *   n >= 4096 and 32 below, nb = 16 b for n >= 32768, 8 b for n >= 16384 and b
 *   below.  b > 0, nb = 0: nb = b.
 *   stream  a cudaStream_t (passed as void*), NULL for the legacy default stream.
 * Must be called with the target device current.  Returns EVD_ERR_INVALID_ARG for
 * n < 0, lda < max(1, n), b < 0, nb < 0, b > 0 && nb % b != 0, or b > 128. */
evd_status_t evd_plan_create(evd_plan_t* plan, int64_t n, int64_t lda, evd_job_t job,
                             evd_prec_t prec, int b, int nb, void* stream);

/* Bytes of device workspace every call on this plan needs (caller allocates,
 * 256-byte aligned).  The same workspace must be passed to the stage calls of one
 * solve, since later stages read what earlier stages left there. */
evd_status_t evd_plan_workspace_size(evd_plan_t plan, size_t* bytes);

/* Plan options: tunables that change how a solve runs, never what it computes
 * beyond the stated accuracy.  Set them after evd_plan_create and before
 * evd_plan_workspace_size and the first stage call (EVD_OPT_SLICES changes the
 * workspace size).  Every option has the default stated here; a value out of its
 * range returns EVD_ERR_INVALID_ARG and leaves the plan unchanged.
 *   EVD_OPT_SLICES        1..8  bfloat16 slices of the back transformation's products
 *                               (default 8 for EVD_FP64, 6 for EVD_SPLIT_BF16).  At 8
 *                               or 6 the fused BC-Back waves run with their 7 digits;
 *                               other values take the batched BC-Back products.
 *   EVD_OPT_SBR_SLICES    1..8  slices of SBR's products, Z formation and trailing
 *                               update (default 8, 7 for EVD_SPLIT_BF16).  The D&C
 *                               merges and the refinement residuals always take 8.
 *   EVD_OPT_REFINE_ITERS  0..8  Ogita-Aishima steps after an EVD_SPLIT_BF16 solve
 *                               (default 2; ignored for EVD_FP64).
 *   EVD_OPT_XE_SLICES     1..8  slices of the refinement's X E product; E holds
 *                               corrections at the error level, so few suffice
 *                               (default 4).
 *   EVD_OPT_BCBACK_FUSED  0, 1  allow the fused BC-Back wave kernel (default 1).
 *   EVD_OPT_BC_KERNEL     0..2  bulge-chasing kernel: 0 band in global memory,
 *                               1 staged in shared memory, 2 staged with the next
 *                               step's rows carried over (default 2).
 *   EVD_OPT_PANEL_CTAS    1..2048  CTAs of the cooperative SBR panel QR (default 64).
 *   EVD_OPT_BC_CTAS_PER_SM 0..4  bulge-chasing sweeps in flight per SM (at most
 *                               what fits; default 0 = two when more sweeps can run
 *                               at once than 2.5 x the SM count, else one).
 *   EVD_OPT_ORDER         -1..1 order of the back transformation in evd_syevd:
 *                               0 conventional (Sec. 2.1.2: X = Q_d, BC-Back, SBR-Back);
 *                               1 reordered (Sec. 3.3: Q_sb = Q_s Q_b I while D&C runs
 *                               on a second stream, then Q = Q_sb Q_d; needs b = 64,
 *                               n >= 1024, the fused BC-Back and n^2 more doubles of
 *                               workspace); -1 (default) reordered from n = 8192 up.
 *                               evd_plan_get_option reports the order a solve takes. */
typedef enum {
  EVD_OPT_SLICES = 0,
  EVD_OPT_REFINE_ITERS = 1,
  EVD_OPT_BCBACK_FUSED = 2,
  EVD_OPT_BC_KERNEL = 3,
  EVD_OPT_PANEL_CTAS = 4,
  EVD_OPT_XE_SLICES = 5,
  EVD_OPT_BC_CTAS_PER_SM = 6,
  EVD_OPT_ORDER = 7,
  EVD_OPT_SBR_SLICES = 8
} evd_option_t;
evd_status_t evd_plan_set_option(evd_plan_t plan, evd_option_t option, int value);
evd_status_t evd_plan_get_option(evd_plan_t plan, evd_option_t option, int* value);

/* The plan's chosen band width and double-blocking width. */
evd_status_t evd_plan_get_blocking(evd_plan_t plan, int* b, int* nb);

/* Stage 1 -- SBR (Sec. 2.1.1, Eq. 1): reduce the lower triangle of A to a band of
 * half-width b.  A is overwritten: its band holds B, below the band it holds the
 * panel Householder vectors (unit diagonal implied); their tau and T factors go to
 * ws.  The band is also packed into ws for the next stage. */
evd_status_t evd_sbr(evd_plan_t plan, double* A, void* ws);

/* Stage 2 -- BC (Sec. 2.1.1, Sec. 4.2): reduce the band in ws to tridiagonal T.
 * d (n) receives the diagonal, e (n-1) the sub-diagonal.  With EVD_VECTORS the BC
 * Householder vectors and tau stay in ws for the back transformation. */
evd_status_t evd_bulge_chase(evd_plan_t plan, void* ws, double* d, double* e);

/* Stage 3 -- divide and conquer (Sec. 1, Sec. 3.3): on entry d (n), e (n-1) hold T;
 * on exit d holds the eigenvalues ascending.  e is destroyed.  If Qd != NULL it
 * receives the n x n eigenvector matrix of T (ldq >= n). */
evd_status_t evd_tridiag_solve(evd_plan_t plan, double* d, double* e, double* Qd, int64_t ldq,
                               void* ws);

/* Stage 4 -- back transformation (Sec. 2.1.2, conventional order): on entry Q holds
 * Q_d; on exit Q = Q_s Q_b Q_d, the eigenvectors of the A given to evd_sbr.  Reads
 * the SBR vectors from the A passed to evd_sbr (still needed: pass it again) and
 * the BC vectors from ws.  With b = 64 and a Q whose base address is 16-byte aligned
 * and ldq even, BC-Back runs the fused wave kernel (Q is held in int64 fixed point in
 * place while it runs); otherwise it runs the batched split products.  Both give
 * FP64-level results. */
evd_status_t evd_back_transform(evd_plan_t plan, const double* A_reduced, void* ws, double* Q,
                                int64_t ldq);

/* The whole path: stages 1-4 (stage 4 only with EVD_VECTORS), plus refinement for
 * EVD_SPLIT_BF16.  A is overwritten (as in LAPACK syevd) -- except for the split
 * mode, which first copies A into ws for the refinement residuals.  w (n) receives
 * the eigenvalues ascending; Q (n x n, ldq) the eigenvectors (may be NULL for
 * EVD_VALUES). */
evd_status_t evd_syevd(evd_plan_t plan, double* A, double* w, double* Q, int64_t ldq, void* ws);

/* Ogita-Aishima refinement (one or more steps) of an approximate eigendecomposition
 * of the symmetric A0 (lower triangle read, lda = the plan's): Q (in/out, ldq) and
 * w (out).  Residual products are FP64-accurate.  Uses ws. */
evd_status_t evd_refine(evd_plan_t plan, const double* A0, double* w, double* Q, int64_t ldq,
                        int iterations, void* ws);

/* Sync the plan's stream and read its device status word.  *info receives a
 * stage-specific index (e.g. the leaf or root that failed), 0 if none.  Clears the
 * status word. */
evd_status_t evd_plan_status(evd_plan_t plan, int* info);

/* Self-test of the bounded device waits (failure detection without a fault).
 * Enqueues on the plan's stream one kernel whose wait never completes and gives up
 * after a short limit (well under a second), through the same wait helpers the
 * solver uses: kind 0 a progress flag that nothing publishes, kind 1 a grid
 * barrier that expects one CTA more than the launch has, kind 2 an mbarrier that
 * nobody arrives at, in a CTA that holds tensor memory (freed before it returns).
 * The kernel returns; evd_plan_status() then reports EVD_ERR_TIMEOUT with info =
 * 9901, 9902 or 9903, clears the status word and the barrier counters, and the
 * plan stays usable.  The paper has no counterpart (the solver's waits are this
 * design's). */
evd_status_t evd_wait_selftest(evd_plan_t plan, int kind);

/* Destroy a plan (syncs its stream first).  NULL is a no-op. */
void evd_plan_destroy(evd_plan_t plan);

/* Static text for a status code. */
const char* evd_status_string(evd_status_t status);

/* ---------------------------------------------------------------------------
 * Batched solve: count independent symmetric problems of uneven size, each with
 * its own A (lower read, overwritten), lda, w, Q, ldq.  Problems are assigned
 * longest first (cost ~ n^3) to up to 8 lanes, each with its own part of ws.  The
 * whole batch runs as one CUDA graph: every solve (a plan each, D&C in its form
 * without host reads) is captured on its lane's stream, the lanes forked from and
 * joined to one stream, and the graph launched once.  The captured graph and its
 * plans are kept until the next call with different arguments: a call with exactly
 * the same arguments launches it again without capturing.  If the driver refuses
 * the capture, the same work runs on live lanes (a stream and host thread each);
 * evd_batched_last_graph() reports which path the last call took.  The work starts
 * after what is already queued on `stream`, `stream` waits for it, and the call
 * returns once every problem has been solved (it reads each problem's status).
 * Arrays n, lda, ldq are HOST arrays of length count; A, w, Q are HOST arrays of
 * DEVICE pointers.  ws/ws_bytes: device workspace of at least
 * evd_batched_workspace_size() bytes (256-byte aligned).  Returns the first error
 * any problem reported.  Not thread-safe against concurrent batched calls on the
 * same graph cache (calls serialize on a lock).
 * ------------------------------------------------------------------------- */
evd_status_t evd_batched_workspace_size(int count, const int64_t* n_host, evd_job_t job,
                                        size_t* bytes);
evd_status_t evd_syevd_batched(int count, const int64_t* n_host, double* const* A_host,
                               const int64_t* lda_host, double* const* w_host,
                               double* const* Q_host, const int64_t* ldq_host, evd_job_t job,
                               void* ws, size_t ws_bytes, void* stream);
/* 1 if the last evd_syevd_batched call ran as a captured graph, 0 if on live lanes. */
int evd_batched_last_graph(void);

/* ---------------------------------------------------------------------------
 * The dense product engine on its own (for tests and benchmarks):
 *   C = alpha * op(A) * op(B) + beta * C, FP64 column-major, op = N or T.
 * slices: 0 = plain FP64 CUDA-core kernel; 1..8 = tensor-core product with that many
 * 7-bit bfloat16 slices per operand (8 = FP64-accurate).  ws must hold
 * evd_gemm_workspace_size() bytes.  Runs on `stream`. */
evd_status_t evd_gemm_workspace_size(int64_t m, int64_t n, int64_t k, int slices, size_t* bytes);
evd_status_t evd_dgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                       const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                       double* C, int64_t ldc, int slices, void* ws, size_t ws_bytes,
                       void* stream);

/* Device status of the stand-alone products (evd_dgemm, evd_dgemm_static): a bounded
 * wait inside the tensor-core product that gave up latches EVD_ERR_TIMEOUT in a status
 * word after the call has returned EVD_OK.  This call synchronizes `stream`, returns the
 * first latched error of evd_dgemm's calls since the last query or, if none, that of
 * the last evd_dgemm_static call on the current device, and clears both words (*info:
 * the location code, may be NULL). */
evd_status_t evd_dgemm_status(void* stream, int* info);

/* ---------------------------------------------------------------------------
 * evd_dgemm without a workspace: the same product as evd_dgemm, with the same
 * arguments minus ws/ws_bytes.  The paper has no counterpart.  It serves callers
 * that cannot allocate device memory or pass a workspace through: a C host with no
 * device allocator, a callback with a fixed signature, or code that must avoid
 * cudaMalloc/cudaFree because they act on the whole device.
 *
 * The scratch is one fixed array in device global memory, EVD_STATIC_SCRATCH_BYTES
 * per device, owned by the library.  The call allocates nothing.  Rules:
 * - A product whose least scratch (that of evd_gemm_workspace_size() with no
 *   split of K; the product lowers its split count to fit) exceeds
 *   EVD_STATIC_SCRATCH_BYTES returns EVD_ERR_WORKSPACE at once, with no device work.
 * - Calls that overlap in time race on the shared array: calls on different
 *   streams, or from different host threads, must not be in flight together.
 *   Calls queued one after another on the same stream are safe.
 * - The first call on each device looks up the array's device address, which
 *   may load the module.  Make that first call outside any stream capture.  The
 *   address is kept for the process: it assumes the device is not reset.
 * Errors: as evd_dgemm; a lookup failure returns EVD_ERR_CUDA.  A device-side
 * timeout is not part of the return value (the call returns before the kernel
 * runs): evd_dgemm_status() reads it. */
#define EVD_STATIC_SCRATCH_BYTES ((size_t)64 << 20)
evd_status_t evd_dgemm_static(char transa, char transb, int64_t m, int64_t n, int64_t k,
                              double alpha, const double* A, int64_t lda, const double* B,
                              int64_t ldb, double beta, double* C, int64_t ldc, int slices,
                              void* stream);

/* Autotuner: time one solve of a seeded symmetric n x n matrix for each candidate
 * (b, nb) with b in {32, 64, 128} and nb in {b, 2b, 4b, 8b, 16b} below n (from
 * n = 32768 on, b = 64 only: the fused BC-Back waves need it), then, for the
 * fastest pair, the bulge chasing with one and with two sweeps in flight per SM
 * (the sweep grouping); the first solve of the call is an untimed warm-up.  Returns
 * the fastest (b, nb) in *b, *nb.  With cache_path != NULL the choice, the sweep
 * grouping included, is kept per (n rounded to a power of two, job, prec) in that
 * JSON file, and a cached entry is returned without timing.  evd_plan_create with
 * b = nb = 0 uses the entry of the file named by the environment variable
 * EVD_AUTOTUNE_CACHE, if there is one.  Allocates its own device memory
 * (cudaMalloc) and runs on the legacy default stream; n <= 65535. */
evd_status_t evd_autotune(int64_t n, evd_job_t job, evd_prec_t prec, const char* cache_path,
                          int* b, int* nb);

/* ---------------------------------------------------------------------------
 * Instrumentation (off by default; used by the benchmark).  When enabled, the
 * library records CUDA events around its launches on the launching stream,
 * grouped by category ("sbr_z/tc_split", "gemm/fp64_simt", "sbr_panel_qr",
 * "bc_chase", "dc_leaf", "dc_merge", "dc_secular", "bc_back", ...), together with
 * the algorithmic flops and bytes of each call.  The library also counts every
 * kernel it launches.  Host-side state, process-wide; not thread-safe across
 * concurrent solves that query it. */
void evd_stats_enable(int on);
void evd_stats_reset(void);
/* Number of kernels launched since the last evd_stats_reset(). */
int64_t evd_launch_count(void);
/* Category names separated by '\n' into buf (capacity cap bytes); returns the count. */
int evd_stats_categories(char* buf, int cap);
/* Device milliseconds (sum over calls, synchronizes the events), algorithmic flops
 * and bytes, and number of calls of one category. */
evd_status_t evd_stats_query(const char* category, double* ms, double* flops, double* bytes, int64_t* calls);

#ifdef __cplusplus
}
#endif
#endif /* EVD_H_ */
