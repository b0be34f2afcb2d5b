/*
 * cvxb300 -- the SCS-style ADMM hot path of "A New Architecture for
 * Optimization Modeling Frameworks" (Wytock, Diamond, Heide, Boyd, 2016) as a
 * C ABI over hand-written CUDA kernels for one B300 (sm_103a).
 *
 * Problem (Section 2.1, problem (1), written with the sign convention of the
 * SCS method that Section 5.2 uses as its solver):
 *
 *     minimise c^T x   subject to   A x + s = b,   s in K
 *
 * with x in R^n, A an m x n linear operator given as a composition of
 * structured operators (Section 3.1: dense, sparse, convolution, Kronecker,
 * diagonal), and K = {0}^z x R_+^l x Q^{q_1} x ... x Q^{q_p} (zero cone,
 * nonnegative orthant, second-order cones Q^q = {(t, u) in R x R^{q-1}:
 * ||u||_2 <= t}), rows of A ordered in that order.
 *
 * Conventions shared by every entry point:
 *   - Return value: CF_OK on success, a negative cf_err otherwise; the
 *     thread-local text of the last failure is cf_last_error().  A solve that
 *     stops without meeting the tolerance still returns CF_OK; its outcome is
 *     cf_info.status.
 *   - Pointers to caller data may point to host memory or to device memory
 *     of the context's GPU (unified addressing tells them apart).  Inputs are
 *     copied into library-owned device memory at creation time; the caller
 *     keeps ownership of its buffers and may free them after the call.
 *   - Output buffers are caller-owned and may be NULL where stated.
 *   - Handles are not thread-safe; distinct handles may be used from
 *     distinct threads.  Operators are reference counted: a composition or a
 *     problem holds references to its parts, so destroying a part after use
 *     is always safe.
 *   - Vectors live on the GPU in float32; reductions, residual norms, the
 *     tau/kappa scalars and the CG stopping test are float64.
 */
#ifndef CVXB300_H
#define CVXB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cf_ctx cf_ctx;
typedef struct cf_op cf_op;
typedef struct cf_problem cf_problem;
typedef struct cf_server cf_server;
typedef int64_t cf_ticket;

typedef enum {
  CF_OK = 0,
  CF_E_INVALID = -1, /* bad argument: sizes, NULL where not allowed, kinds */
  CF_E_OOM = -2,     /* device or host allocation failed */
  CF_E_CUDA = -3,    /* a CUDA runtime call failed (message in cf_last_error) */
  CF_E_BUSY = -4,    /* server queue full; nothing was enqueued */
  CF_E_TIMEOUT = -5, /* serve_wait: result not ready within the timeout */
  CF_E_STATE = -6    /* handle in the wrong state (e.g. unknown ticket) */
} cf_err;

typedef enum {
  CF_SOLVED = 0,     /* residuals and gap below eps (x, y, s returned) */
  CF_INFEASIBLE = 1, /* certificate y returned (b^T y = -1, A^T y ~ 0, y in K*) */
  CF_UNBOUNDED = 2,  /* certificate x, s returned (c^T x = -1, A x + s ~ 0) */
  CF_MAX_ITERS = 3,  /* iteration limit; last iterate returned */
  CF_NUMERICAL = 4,  /* NaN/Inf appeared in the iterates */
  CF_CANCELLED = 5   /* serving: request dropped before it ran */
} cf_status;

typedef enum { CF_FP32 = 0, CF_BF16 = 1, CF_FP8_E4M3 = 2 } cf_prec;

typedef enum {
  CF_VSTACK = 0,    /* [P1; P2; ...]          parts share n            */
  CF_HSTACK = 1,    /* [P1, P2, ...]          parts share m            */
  CF_BLOCKDIAG = 2, /* diag(P1, P2, ...)                               */
  CF_PRODUCT = 3,   /* P1 P2 ... Pk           P_i.n == P_{i+1}.m       */
  CF_SUM = 4,       /* P1 + P2 + ...          equal shapes             */
  CF_SCALE = 5,     /* alpha * P1             (k == 1)                 */
  CF_ADJOINT = 6,   /* P1^T                   (k == 1)                 */
  CF_KRON = 7       /* P1 (x) P2, row-major vec: (A (x) B) vec(X) =
                       vec(A X B^T); both parts dense FP32             */
} cf_compose_kind;

/* Cone K: z zero rows, l nonnegative rows, then nq second-order cones of
 * sizes q[0..nq-1] (each >= 1; the first row of each block is t). */
typedef struct {
  int64_t z;
  int64_t l;
  const int64_t* q;
  int64_t nq;
} cf_cone;

typedef struct {
  double eps;             /* stop when pri, dual and gap residuals <= eps (1e-4) */
  double eps_infeas;      /* certificate threshold (1e-4) */
  double alpha;           /* relaxation parameter in (0, 2) (1.5) */
  int32_t max_iters;      /* ADMM iteration limit (100000) */
  int32_t check_interval; /* residual check every this many iterations (10) */
  int32_t cg_max_iters;   /* CG step cap per ADMM iteration (50) */
  int32_t cg_fixed_iters; /* > 0: exactly this many CG steps per iteration,
                             no tolerance test (trajectory mode) (0) */
  double cg_tol_rel;      /* CG stops when ||r|| <= max(cg_tol_min,            */
  double cg_tol_exp;      /*   cg_tol_rel ||rhs|| (k+1)^-cg_tol_exp) (1, 1.5)  */
  double cg_tol_min;      /*   at ADMM iteration k (1e-9)                      */
  int32_t setup_cg_max_iters; /* CG cap for g = M^{-1} h at setup (2000) */
  double setup_cg_tol;        /* relative CG tolerance at setup (1e-7) */
  int32_t host_loop;  /* 0: the whole solve is one CUDA graph whose loops run on
                         the device (default).  1: the host launches the same
                         kernels and reads each loop decision back (slower; for
                         profilers that do not see kernels inside graph
                         conditional nodes, and for debugging). */
  int32_t engine;     /* cf_engine: which of the two solver programs runs the
                         iterations (CF_ENGINE_AUTO). */
} cf_settings;

/* The solver has three programs for the same iteration:
 *  - the graph engine: one CUDA graph per solve whose kernels each spread
 *    one step over the whole GPU (large problems);
 *  - the team engine: one persistent kernel in which a team of CTAs (one CTA,
 *    or a thread-block cluster) runs a problem's whole solve, synchronising
 *    with barriers instead of kernel boundaries, and a batch is one launch
 *    whose teams take problems from a longest-first work queue (small and
 *    medium problems, batches, serving);
 *  - the grid engine: the team engine's solve with every SM in the team
 *    (one cooperative launch, one CTA per SM, grid-wide barriers and
 *    reductions): one large problem's whole solve in one launch.
 * All compute the same iteration; their float32 rounding differs (other
 * reduction partitions).  The team and grid engines support operator trees
 * of dense, CSR, 1-D convolution (direct sums up to 2048 taps, or overlap-save
 * FFTs), diagonal and zero leaves under vstack, hstack, blockdiag, sum, scale
 * and adjoint, with at most 4 second-order cones and dense leaves of at most
 * 16384 columns. */
typedef enum {
  CF_ENGINE_AUTO = 0,  /* team engine when the problem is supported and one
                          operator pass is at most the schedule's
                          auto_max_bytes (batch_max_bytes inside
                          solve_batch); graph engine otherwise */
  CF_ENGINE_GRAPH = 1, /* always the graph engine */
  CF_ENGINE_TEAM = 2,  /* always the team engine (CF_E_INVALID if the
                          problem is not supported) */
  CF_ENGINE_GRID = 3   /* the grid engine for single solves (CF_E_INVALID if
                          the problem is not supported); inside solve_batch it
                          means CF_ENGINE_TEAM and in serving CF_ENGINE_AUTO.
                          Each grid-wide barrier wait is bounded: if one gives
                          up, the solve returns CF_E_CUDA. */
} cf_engine;

/* Launch schedule of the team engine, held by the context.  A problem's
 * iterates depend on the schedule it ran with (it fixes the reduction
 * partitions), never on the other problems of a batch. */
typedef struct {
  int32_t cluster;         /* CTAs per cluster team: 1, 2, 4 or 8 (4) */
  int32_t threads;         /* threads per CTA: 256, 512 or 1024 (512) */
  int32_t csr_nnz_per_lane;/* CSR rows get the fewest lanes (a power of two,
                              1..32) that hold the average row at this many
                              nonzeros per lane (16) */
  int32_t ctas_per_sm;     /* team CTAs that share an SM: 1, 2 (threads <= 512)
                              or 4 (threads 256) -- the registers of a thread
                              shrink to fit (1) */
  double team_bytes;       /* problems whose operator pass reads at least this
                              many bytes run on a whole cluster team; smaller
                              ones on one CTA (256e3) */
  double auto_max_bytes;   /* CF_ENGINE_AUTO limit for single and served solves
                              (1e6: above it the graph engine's whole-GPU
                              passes outrun a cluster team) */
  double batch_max_bytes;  /* CF_ENGINE_AUTO limit inside solve_batch (48e6: the
                              batch's other problems keep the SMs busy) */
} cf_schedule;

typedef struct {
  int32_t status;          /* cf_status */
  int32_t iters;           /* ADMM iterations run */
  int64_t cg_iters_total;  /* CG steps over all iterations */
  int32_t checks;          /* residual checks run */
  int32_t setup_cg_iters;  /* CG steps at setup (0 if setup was cached) */
  double pri_res, dual_res, gap; /* at the last check (see eps) */
  double pobj, dobj;       /* c^T x and -b^T y at the returned point */
  double tau, kappa;       /* embedding scalars at exit */
  int64_t setup_ns;        /* host time preparing the setup (0 if cached) */
  int64_t solve_ns;        /* wall time from launch to completion (includes
                              the setup's GPU time when it ran) */
  int64_t kernel_launches; /* kernels this call ran on the GPU */
  int64_t queue_ns;        /* serving: time from serve_submit to launch */
  int64_t device_ns;       /* team engine: device time of this problem's
                              solve inside its launch (0 on the graph engine) */
} cf_info;

/* Fill *s with the defaults listed above. */
void cf_settings_default(cf_settings* s);

/* ----------------------------------------------------------------- context
 * A context binds a CUDA device and a stream.  cuda_stream (a cudaStream_t)
 * may be NULL: the context then creates and owns a non-blocking stream.  Work
 * submitted through the context is ordered after earlier work on that
 * stream, and blocking calls return after their work finished. */
cf_err cf_ctx_create(int device, void* cuda_stream, cf_ctx** out);
void cf_ctx_destroy(cf_ctx* ctx);
/* Streaming multiprocessor count of the context's device. */
int cf_ctx_sm_count(const cf_ctx* ctx);

/* ---------------------------------------------------------------- operators
 * Leaves (Section 3.1 structured linear operators).  Each leaf has a
 * forward (A x) and an adjoint (A^T y) kernel (Section 4.1: adjoints of
 * linear maps are derived, not stored as transposed matrices, except for
 * CSR, which keeps its transpose for a deterministic adjoint). */

/* Dense m x n, row-major float32 input.  storage: CF_FP32 keeps it;
 * CF_BF16 rounds every entry to bfloat16 (nearest, ties to even);
 * CF_FP8_E4M3 stores e4m3 codes (nearest, ties to even, saturating at 448)
 * of a_ij / s_i with per-row scale s_i = max_j |a_ij| / 448 (1 for a zero
 * row).  The stored values define the operator. */
cf_err cf_op_dense(cf_ctx* ctx, int64_t m, int64_t n, const float* A, cf_prec storage,
                   cf_op** out);

/* CSR m x n with nnz entries (rowptr[m] == nnz, 0 <= col < n, int32).
 * storage CF_FP32 or CF_BF16 (values rounded as for dense). */
cf_err cf_op_csr(cf_ctx* ctx, int64_t m, int64_t n, int64_t nnz, const int32_t* rowptr,
                 const int32_t* col, const float* val, cf_prec storage, cf_op** out);

/* Full 1-D convolution with a length-L kernel: (k * x)[i] = sum_l k[l] x[i-l],
 * an (n + L - 1) x n operator (Section 5.3's c * x).  Same as
 * cf_op_conv1d_method with CF_CONV_AUTO. */
cf_err cf_op_conv1d(cf_ctx* ctx, int64_t n, const float* kernel, int64_t L, cf_op** out);

/* How a 1-D convolution leaf is evaluated: the direct sum (FP32 FMAs over
 * the taps), or overlap-save FFTs of 4096 points in FP32 (Section 2's
 * FFT-based convolution; taps padded to a multiple of 16 must number at most
 * 2048, else CF_E_INVALID).  CF_CONV_AUTO takes the FFT for 256 to 2048
 * padded taps.  The FFT's error is bounded in the 2-norm of each
 * 4096-sample input segment rather than entry by entry. */
typedef enum { CF_CONV_AUTO = 0, CF_CONV_DIRECT = 1, CF_CONV_FFT = 2 } cf_conv_method;
cf_err cf_op_conv1d_method(cf_ctx* ctx, int64_t n, const float* kernel, int64_t L, int32_t method,
                           cf_op** out);

/* Full 2-D convolution of an h x w image (row-major) with a kh x kw kernel:
 * Y[a, b] = sum_{p,q} K[p, q] X[a-p, b-q], output (h+kh-1) x (w+kw-1). */
cf_err cf_op_conv2d(cf_ctx* ctx, int64_t h, int64_t w, const float* kernel, int64_t kh,
                    int64_t kw, cf_op** out);

/* n x n diagonal; d == NULL gives the identity. */
cf_err cf_op_diag(cf_ctx* ctx, int64_t n, const float* d, cf_op** out);

/* m x n zero operator. */
cf_err cf_op_zero(cf_ctx* ctx, int64_t m, int64_t n, cf_op** out);

/* Composition of k >= 1 parts (see cf_compose_kind); alpha is used by
 * CF_SCALE only.  The result references its parts. */
cf_err operator_compose(cf_ctx* ctx, cf_compose_kind kind, cf_op* const* parts, int32_t k,
                        double alpha, cf_op** out);

/* Kronecker product A (x) B (Section 3.1 lists it among the structured
 * operators; the paper's image example uses it for separable kernels):
 * (mA mB) x (nA nB), row-major vec: (A (x) B) vec(X) = vec(A X B^T), applied
 * as two GEMMs without forming the product.  The same operator as
 * operator_compose(CF_KRON, {A, B}); both parts dense FP32 leaves
 * (CF_E_INVALID otherwise).  The result references A and B. */
cf_err cf_op_kron(cf_ctx* ctx, cf_op* A, cf_op* B, cf_op** out);

/* Drop the caller's reference. NULL is ignored. */
void cf_op_destroy(cf_op* op);

cf_err cf_op_shape(const cf_op* op, int64_t* m, int64_t* n);

/* y = A x (adjoint == 0, x has n entries, y has m) or y = A^T x (adjoint != 0,
 * x has m, y has n); float32, host or device pointers; blocks until done. */
cf_err cf_op_apply(cf_op* op, int32_t adjoint, const float* x, float* y);

/* Device-only, allocation-free form of cf_op_apply for callers that manage
 * their own buffers and stream: enqueue y = alpha * op(x) + (accumulate ? y :
 * 0) on `stream` (a cudaStream_t; NULL = the context stream) and return
 * without waiting.  x, y: device float32; workspace: device memory of at least
 * cf_op_workspace_bytes(op, adjoint) bytes (may be NULL when that is 0),
 * which must not be in use by other work on the GPU until this call's work
 * finished.  x must not overlap y. */
cf_err cf_op_apply_async(cf_op* op, int32_t adjoint, float alpha, const float* x, float* y,
                         int32_t accumulate, void* workspace, void* stream);
cf_err cf_op_workspace_bytes(const cf_op* op, int32_t adjoint, size_t* bytes);

/* Size of the static scratch array behind cf_op_apply_static (16 MiB). */
#define CF_STATIC_SCRATCH_BYTES (16u << 20)

/* Allocation-free apply, for callers that may not allocate GPU memory at
 * all: code that runs inside a framework or server whose allocator owns all
 * device memory (a raw cudaMalloc would bypass its accounting or fail against
 * its reservation), and latency-critical loops where cudaMalloc/cudaFree would
 * stall or synchronize the device.  The paper has no counterpart; this is an
 * interface convenience.
 *
 * Same result as cf_op_apply_async (y = alpha * op(x) + (accumulate ? y : 0),
 * x and y device float32, enqueued on `stream`, NULL = the context stream,
 * returns without waiting), but the operator's scratch (the dense adjoint's
 * per-row-block partial sums, product and Kronecker intermediates) comes from
 * one file-scope device array of CF_STATIC_SCRATCH_BYTES that every GPU which
 * loads the library holds until the process exits.  No device or host memory
 * is allocated.  Operators needing more scratch than that are rejected with
 * CF_E_INVALID.  The first call on a device looks up the array's device
 * address (once per device), so make that first call before any stream
 * capture.  All calls share the one array: calls whose GPU work overlaps
 * (different streams, or different host threads) race and give wrong results;
 * serialize them.  Each call writes every scratch element before reading it,
 * so the contents left by the previous call do not matter.  x must be ready on
 * `stream`: when x was written on another stream, the caller orders the two
 * (an event, or passing the producing stream here).  An error already pending
 * on the calling thread is returned as CF_E_CUDA and left in place.  The
 * array's device address is cached per device for the life of the process:
 * do not use this entry point after cudaDeviceReset or a re-creation of the
 * device's primary context. */
cf_err cf_op_apply_static(cf_op* op, int32_t adjoint, float alpha, const float* x, float* y,
                          int32_t accumulate, void* stream);

/* Copy a dense leaf's stored operand out: codes receives m*n entries
 * (float32 for CF_FP32, bfloat16 bit patterns for CF_BF16, e4m3 bytes for
 * CF_FP8_E4M3), row_scale receives m float32 scales (CF_FP8_E4M3 only; may be
 * NULL otherwise).  Host or device pointers. */
cf_err cf_op_dense_stored(const cf_op* op, void* codes, float* row_scale);

/* ------------------------------------------------------------------ problem
 * Cone program over operator A (m x n): b (m) and c (n) float64, K as above
 * with z + l + sum q == m.  The problem references A. */
cf_err cone_problem_create(cf_ctx* ctx, const cf_op* A, const double* b, int64_t m,
                           const double* c, int64_t n, const cf_cone* K, cf_problem** out);
void cf_problem_destroy(cf_problem* p);

/* Run the SCS iteration (Section 5.2) on the GPU until the residuals meet
 * settings->eps (checked every check_interval iterations), a certificate is
 * found, or max_iters is reached.  settings may be NULL (defaults).
 * x (n), y (m), s (m): float64 outputs, each may be NULL.  warm_uv: NULL or
 * 2(n+m+1) float64 values u = (x, y, tau), v = (r, s, kappa) to start from
 * (default u = v = (0, 0, 1)).  uv_out: NULL or 2(n+m+1) float64 receiving
 * the final u, v.  info may be NULL.  The first solve of a problem runs its
 * setup (g = M^{-1} h by CG), later solves reuse it.  Blocks until done. */
cf_err solve(cf_problem* p, const cf_settings* settings, double* x, double* y, double* s,
             const double* warm_uv, double* uv_out, cf_info* info);

/* Solve count problems concurrently: the team-engine problems in one
 * persistent launch (longest first), each graph-engine problem on a CUDA
 * stream of its own.  xs/ys/ss may be
 * NULL or arrays of count pointers (entries may be NULL); infos may be NULL.
 * Returns the first error; every problem is attempted. */
cf_err solve_batch(cf_problem* const* probs, int32_t count, const cf_settings* settings,
                   double* const* xs, double* const* ys, double* const* ss, cf_info* infos);

/* Matrix-free data equilibration (Section 3: forward and adjoint
 * evaluations suffice to precondition a problem, after stochastic matrix-free
 * equilibration).  Finds positive diagonal scalings D (rows; one factor per
 * second-order cone block) and E (columns) with `iters` Ruiz steps, each
 * estimating the squared row and column norms of D A E from `probes` random
 * sign vectors (SplitMix64 of `seed`, counter-based); then scales b and c to
 * unit norm (sigma, rho).  Later solves iterate on D A E, sigma D b, rho E c
 * and stop on, and return, the original problem's residuals and point
 * (warm-start / uv vectors are in the scaled coordinates).  The problem's
 * setup is redone at its next solve.  iters in [0, 100], probes in
 * [1, 1024]; CF_E_STATE if the problem is already equilibrated. */
cf_err cone_problem_equilibrate(cf_problem* p, int32_t iters, int32_t probes, uint64_t seed);

/* Mixed-precision refinement (the BF16/FP8 accuracy reading beside Section
 * 5.2's lasso operands): the problem keeps A as its instance and, from the
 * next solve on, every CG step of the ADMM iterations applies inner -- an
 * operator of A's shape, normally A stored in BF16 or FP8 -- instead of A.
 * The carried A z_x and A^T A z_x then advance by inner's increments; the
 * right-hand side w_x - A^T w_y, the setup (g = M^{-1} h), the residual and
 * certificate tests, and the exact recomputation of the carried vectors
 * every 50 iterations keep applying A, so the iteration's fixed points are
 * those of the problem with A.  inner is referenced, not copied (it may be
 * destroyed by the caller afterwards); NULL turns refinement off.  An
 * equilibrated problem scales inner by the same D, E (also when it is
 * equilibrated later).  Problems with an inner operator run on the graph
 * engine only (CF_ENGINE_AUTO picks it; CF_ENGINE_TEAM is CF_E_INVALID).
 * CF_E_INVALID: NULL p, inner's shape differs from A's, or inner belongs to
 * another context. */
cf_err cone_problem_set_inner(cf_problem* p, const cf_op* inner);

/* The equilibration of a problem: D (m floats), E (n floats) -- host or
 * device buffers, may be NULL -- and sigma, rho (all 1 without
 * equilibration). */
cf_err cf_problem_scaling(const cf_problem* p, float* D, float* E, double* sigma, double* rho);

/* The team engine's view of a problem: *supported = 1 when the team engine
 * can run it (else 0, and why -- when not NULL -- receives the reason,
 * NUL-terminated, at most why_len bytes); *pass_bytes = the bytes (and
 * flop-equivalents of convolutions) one forward operator pass reads, the size
 * that cf_schedule's team_bytes and auto_max_bytes are compared with.  Any
 * output pointer may be NULL. */
cf_err cf_problem_team_info(const cf_problem* p, int32_t* supported, double* pass_bytes, char* why,
                            size_t why_len);

/* The context's team-engine schedule (see cf_schedule).  Setting it
 * validates every field (CF_E_INVALID) and applies to later solves. */
cf_err cf_ctx_get_schedule(const cf_ctx* ctx, cf_schedule* out);
cf_err cf_ctx_set_schedule(cf_ctx* ctx, const cf_schedule* sched);

typedef struct {
  int32_t candidates;  /* schedules timed */
  int32_t problems;    /* team-engine problems of the batch that were timed */
  double seconds;      /* wall time of the tuning */
  double default_ms;   /* batch time of the schedule held before tuning */
  double best_ms;      /* batch time of the chosen schedule */
  cf_schedule best;    /* now held by the context */
} cf_tune_info;

/* Autotuner of the team engine (a schedule search; the paper has no
 * counterpart -- it solves one problem at a time): times `iters` ADMM
 * iterations (2 CG steps each, no residual checks) of the batch's
 * team-engine problems under candidate schedules -- threads per CTA x CTAs
 * per SM and CSR lanes per row first (24), then the cluster size and the size
 * threshold between cluster teams and one-CTA teams (9) -- and stores the
 * fastest in the problems' context.  The problems must share one context; their iterates are
 * overwritten and their setup is redone at the next solve.  info may be
 * NULL. */
cf_err solve_batch_tune(cf_problem* const* probs, int32_t count, int32_t iters, cf_tune_info* info);

/* Regularized least squares (Section 5.1): x = (lam I + A^T A)^{-1} rhs by CG
 * from x's initial contents, stopping when ||r|| <= tol ||rhs|| (the paper's
 * rule) or after max_iters steps.  rhs, x: float32, n entries, host or
 * device.  iters / res_norm may be NULL. */
cf_err cg_solve(cf_op* A, double lam, const float* rhs, float* x, int32_t max_iters, double tol,
                int32_t* iters, double* res_norm);

/* ------------------------------------------------------------------ serving
 * A server runs a host thread that admits submitted solves while their
 * device memory fits in mem_budget_bytes and fewer than max_slots run, and
 * runs admitted solves concurrently on the GPU (continuous batching: a new
 * request starts as soon as a slot and memory are free, while others are
 * mid-solve). */
cf_err serve_create(cf_ctx* ctx, size_t mem_budget_bytes, int32_t max_slots, cf_server** out);
/* Non-blocking: enqueue a solve of p (settings copied; NULL = defaults).
 * Returns CF_E_BUSY without enqueuing when the queue holds 4096 requests, and
 * CF_E_INVALID when p alone exceeds the memory budget. */
cf_err serve_submit(cf_server* srv, cf_problem* p, const cf_settings* settings, cf_ticket* out);
/* Wait up to timeout_ns (< 0: forever) for a ticket; on success copy its
 * results (any pointer may be NULL) and retire the ticket. */
cf_err serve_wait(cf_server* srv, cf_ticket t, int64_t timeout_ns, double* x, double* y, double* s,
                  cf_info* info);
/* Stop admitting, cancel queued requests, wait for running ones, free. */
void serve_destroy(cf_server* srv);

/* ------------------------------------------------------------ measurement
 * The paper has no counterpart; this is a measurement helper.  Fused
 * multiply-add rate of the context's GPU in float32 (fp64 == 0) or float64
 * (fp64 != 0), in flop/s (an FMA counts 2): a full-occupancy grid of
 * independent FMA chains, timed with CUDA events on the context stream (best
 * of 3 launches of ~10 ms after one warm-up).  It is the measured denominator
 * of the ALU-bound rooflines (the convolution leaves).  Blocks until done;
 * allocates a few KB of stream-ordered scratch. */
cf_err cf_measure_fma_rate(cf_ctx* ctx, int32_t fp64, double* flops_per_s);

/* Text of the calling thread's last error ("" if none). */
const char* cf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CVXB300_H */
