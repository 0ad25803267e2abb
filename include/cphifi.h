/*
 * cphifi.h — C ABI of the GB300 solver for the unaligned infinite-dimensional
 * (kernel-mode) CP-HIFI subproblem.
 *
 * The operation: Brust & Kolda, "Fast and Accurate CP-HIFI Tensor
 * Decompositions Exploiting Kronecker Structure", §4.  For one kernel mode
 * with kernel matrix K (n x n, symmetric PSD), the other modes' factor
 * matrices A_m (n_m x r), and q observations (i_l, i_1^l, .., i_d^l, t_l),
 * the library solves the rho-regularised normal equations of §4.1
 * (Eq. unaligned-infinite-1)
 *
 *     [F'F + lambda (I_r (x) K) + rho I_rn] vec(W) = vec(K B)
 *
 * with F(l,:) = Zhat(l,:) (x) K(i_l,:) (Eqs. zhat, khat, F) and B the sparse
 * MTTKRP (row i of B = sum over observations with i_l = i of t_l Zhat(l,:)),
 * by preconditioned conjugate gradients with the matrix-free product of
 * §4.4.1 (Eqs. vl, yhat1) and the Kronecker-eigen preconditioner of §4.4.2
 * (Eqs. precon, fx).
 *
 * Conventions shared by every call:
 *  - Matrices are column-major (Fortran order).  vec() stacks columns, so an
 *    n x r matrix X is the vector x[i + n*j] = X(i,j).
 *  - Indices are 0-based int32.
 *  - `mem` arguments say where the pointers of that call live:
 *    CPHIFI_MEM_HOST (pageable or pinned host memory) or CPHIFI_MEM_DEVICE
 *    (device memory of the context's GPU).  Device pointers must be 8-byte
 *    aligned.
 *  - The caller owns every buffer it passes; the library copies what it needs
 *    before the call returns.  Handles are released by the matching destroy.
 *  - Every call is synchronous with respect to the host unless stated
 *    otherwise: when it returns, outputs are written.
 *  - Calls return a cphifi_status; the human-readable reason of the last
 *    failure of a context is cphifi_last_error(ctx).  No C++ exception
 *    crosses this boundary.  A context is not thread-safe: use one context per
 *    host thread.
 */
#ifndef CPHIFI_H
#define CPHIFI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cphifi_status {
  CPHIFI_OK = 0,
  CPHIFI_E_INVALID_ARG = 1,   /* shape, index range, non-finite value, rho <= 0 */
  CPHIFI_E_OOM = 2,           /* device allocation failed */
  CPHIFI_E_ADMISSION = 3,     /* the footprint exceeds the context's HBM budget */
  CPHIFI_E_NOT_CONVERGED = 4, /* max_iter reached; W and stats are still written */
  CPHIFI_E_BREAKDOWN = 5,     /* p'Ap <= 0 or a non-finite CG scalar */
  CPHIFI_E_DEVICE = 6,        /* a CUDA call failed */
  CPHIFI_E_TIMEOUT = 7,       /* cphifi_wait ran out of time */
  CPHIFI_E_UNSUPPORTED = 8    /* a valid request this build does not implement */
} cphifi_status;

enum { CPHIFI_MEM_HOST = 0, CPHIFI_MEM_DEVICE = 1 };

/* Arithmetic of the PCG operator (§4.4.1 product).  CG vectors, scalars and
 * reductions are FP64 in all modes.
 *  FP64          : every step in FP64 (FP64 FMA units).
 *  MIXED_FP32    : operator in FP32 (FP32 products, FP32 gather-dot/scatter);
 *                  every k_replace iterations an FP64-accurate true residual
 *                  is formed, and only it decides convergence.  PCG restarts
 *                  from it (p = M^{-1} r) when the recurrence residual has met
 *                  the tolerance or fallen below half the true residual (the
 *                  low-precision operator's error then dominates), and
 *                  otherwise runs on with its Krylov space intact.
 *  MIXED_TF32    : as MIXED_FP32 with the two n x n products on the tensor
 *                  cores in TF32 (FP32 accumulate).
 *  MIXED_BF16    : as MIXED_TF32 with BF16 operands.
 *  MIXED_TF32X3  : as MIXED_TF32 with each operand split into two TF32 parts
 *                  (hi + lo) and the product accumulated as hi*hi + hi*lo +
 *                  lo*hi on the tensor cores: near-FP32 accuracy.
 *  MIXED_BF16X3  : as MIXED_FP32 with the two n x n products on the tensor
 *                  cores from the first 3 of the 8-bit BF16 slices that
 *                  FP64_EMULATED uses (each operand row / column scaled to
 *                  its largest entry; the slice products of index sum <= 2,
 *                  summed exactly): per term a few 2^-24 of the scales,
 *                  FP32-level accuracy.
 *                  Needs the kernel's slices (else CPHIFI_E_UNSUPPORTED).
 *  FP64_EMULATED : every step FP64-accurate without the FP64 units: the
 *                  gather-dot/scatter in double-float arithmetic (pairs of
 *                  FP32 numbers, 48-bit significand, error-free TwoSum /
 *                  TwoProd transforms), the two n x n products on the tensor
 *                  cores from 7 BF16 slices of each operand (error-free
 *                  splitting; the leading slice products are summed exactly),
 *                  or in double-float arithmetic when the kernel has no
 *                  slices (no tensor cores, or no room in the HBM budget).
 * In every mode but FP64, the FP64-accurate steps (right-hand side, true
 * residuals, W = U_K Wbar) use this arithmetic: on GB300 the FP32 units and
 * the tensor cores are far faster than the FP64 units.                      */
typedef enum cphifi_precision {
  CPHIFI_FP64 = 0,
  CPHIFI_MIXED_FP32 = 1,
  CPHIFI_MIXED_TF32 = 2,
  CPHIFI_MIXED_BF16 = 3,
  CPHIFI_FP64_EMULATED = 4,
  CPHIFI_MIXED_TF32X3 = 5,
  CPHIFI_MIXED_BF16X3 = 6
} cphifi_precision;

/* Problem-creation flags. */
#define CPHIFI_OBS_SORTED 0x1u  /* kidx is non-decreasing: skip the device sort */
#define CPHIFI_NEED_FP64 0x2u   /* build the FP64 operator data (FP64 mode)      */
#define CPHIFI_NEED_LOWP 0x4u   /* build the hi/lo FP32 operator data (other
                                   modes); neither flag: both are built; a mode
                                   whose data is missing builds it on first use */
#define CPHIFI_KEEP_OBS 0x8u    /* keep the observation lists on the device in
                                   sorted order: needed by the alternating-fit
                                   calls (set_factors, update_factor, fit) */
#define CPHIFI_VALS_F32 0x10u   /* the observed values are FP32 (float), not
                                   FP64 (double): half the bytes to copy; they
                                   are widened to FP64 on the device, and the
                                   solve is then exact for those values    */

typedef struct cphifi_params {
  double lambda;      /* RKHS regularisation, >= 0 (§2)                       */
  double rho;         /* extra ridge making the system definite, > 0 (§4.1)   */
  double tol;         /* stop when ||b - A w|| / ||b|| <= tol                 */
  int32_t max_iter;   /* bound on PCG iterations over all restarts            */
  int32_t precision;  /* cphifi_precision                                      */
  int32_t k_replace;  /* mixed: FP64 true-residual check every k (>= 1)      */
  int32_t check_every;/* FP64: iterations between host convergence polls (>=1)*/
  int32_t profile;    /* 1: time every n x n product and gather-dot/scatter  */
  int32_t gram;       /* how the product forms Yhat1 (Eq. yhat1), 0, 1 or 2:
                         0: every product streams Zhat (Eqs. vl, yhat1);
                         1: the PCG iterations apply the per-index Gram
                            blocks C_i = sum_{i_l = i} Zhat(l,:)'Zhat(l,:)
                            instead (Yhat1(i,:) = C_i Xhat(i,:)', n r^2 values
                            read per product instead of q r), built once per
                            problem on first use -- FP32 for the mixed modes,
                            FP64-accurate otherwise -- and kept until the
                            factors change; the FP64-accurate checks of the
                            mixed modes still stream Zhat;
                         2: as 1, and the FP64-accurate checks (true
                            residuals) also apply FP64-accurate blocks.      */
} cphifi_params;

typedef struct cphifi_stats {
  int32_t status;            /* cphifi_status of the solve                    */
  int32_t iterations;        /* PCG iterations (operator applications)        */
  int32_t true_residuals;    /* FP64 true-residual evaluations                */
  int32_t restarts;          /* refinement restarts (mixed)                   */
  double rel_residual;       /* final ||b - A w||/||b|| (FP64, true residual) */
  double rel_residual_recurrence;
  double setup_ms;           /* problem creation (copies, sort, Zhat, eig V)  */
  double solve_ms;           /* the PCG solve incl. RHS and the final W       */
  /* profile = 1 only: summed CUDA-event durations on the launch stream */
  double gds_ms;             /* gather-dot/scatter launches, operator arith.  */
  int32_t gds_launches;
  int32_t gemm_launches;     /* n x n products, operator arithmetic           */
  double gemm_ms;
  double gds64_ms;           /* FP64 launches used by true residuals (mixed)  */
  int32_t gds64_launches;
  int32_t gemm64_launches;
  double gemm64_ms;
  int64_t kernel_launches;   /* every kernel this solve launched              */
  int64_t setup_launches;    /* kernels launched by the problem's creation    */
  double rhs_ms;             /* CUDA-event time: right-hand side and start     */
  double iter_ms;            /* CUDA-event time: the PCG loop (operator,
                                updates, preconditioner, FP64 true residuals
                                and restarts), i.e. the iteration phase        */
  double final_ms;           /* CUDA-event time: W = U_K Wbar and its copy    */
  double queue_ms;           /* submitted requests: wait for admission (host) */
  double graph_build_ms;     /* host time spent building this solve's CUDA graphs */
} cphifi_stats;

typedef struct cphifi_ctx cphifi_ctx;
typedef struct cphifi_kernel cphifi_kernel;
typedef struct cphifi_problem cphifi_problem;

/* ---- context --------------------------------------------------------------
 * cphifi_ctx_create: bind to CUDA device `device`, create the library's
 * stream, and cap the device memory this context may hold at
 * hbm_budget_bytes (0 = no cap).  Writes the handle to *out. */
int cphifi_ctx_create(cphifi_ctx** out, int device, size_t hbm_budget_bytes);
int cphifi_ctx_destroy(cphifi_ctx* ctx);
/* Order the library's work after, and the caller's later work after the
 * library's, on `stream` (a cudaStream_t; NULL = the legacy default stream).
 * Each call records an event on `stream`, waits on it, and records its own
 * completion back onto `stream`. */
int cphifi_ctx_set_stream(cphifi_ctx* ctx, void* stream);
/* Bytes of device memory the context holds now. */
size_t cphifi_ctx_bytes_in_use(const cphifi_ctx* ctx);
const char* cphifi_last_error(const cphifi_ctx* ctx);
const char* cphifi_status_string(int status);

/* ---- kernel matrix (one-time per K; §3.2 Eq. eigK, reused across the
 * alternating optimisation) -------------------------------------------------
 * n      : kernel-mode size.
 * K      : n x n symmetric PSD kernel matrix, column-major; may be NULL when
 *          UK and DK are given (the solver works in K's eigenbasis).
 * UK, DK : K = UK diag(DK) UK' with UK orthogonal (n x n, column-major,
 *          column j = eigenvector j) and DK the n eigenvalues.  Pass both, or
 *          neither: then the library computes them from K on the device
 *          (FP64 cyclic two-sided Jacobi with a parallel ordering, this
 *          library's own kernels; the lower triangle of K is read;
 *          n <= 4096, larger n gives CPHIFI_E_UNSUPPORTED: pass UK and DK).
 *          Tiny negative eigenvalues are clamped to 0 inside the
 *          preconditioner only.
 * The library keeps FP64 and FP32 copies of UK on the device and, where the
 * tensor cores are available and the context's HBM budget has room, the
 * TF32/BF16 operand copies of the tensor-core modes and 7 BF16 slices of UK
 * and UK' for the FP64-accurate products (about 28 + 28 bytes per entry). */
int cphifi_kernel_create(cphifi_ctx* ctx, int64_t n, const double* K,
                         const double* UK, const double* DK, int mem,
                         cphifi_kernel** out);
/* Fails with CPHIFI_E_INVALID_ARG while a submitted request that uses the
 * kernel has not completed. */
int cphifi_kernel_destroy(cphifi_kernel* kern);
/* ---- kernel matrices from design points (§2: k(x_i, x_j) on the kernel
 * mode's points) --------------------------------------------------------------
 * cphifi_kernel_create_points: the kernel handle of K(i, j) = k(x_i, x_j)
 * for n points x (row-major n x dim, memory kind mem), built on the device
 * in FP64 and decomposed there (as cphifi_kernel_create with K alone, so
 * n <= 4096).  kind: CPHIFI_KERNEL_GAUSSIAN, k = exp(-|x - y|^2 / (2 s^2)),
 * or CPHIFI_KERNEL_MATERN32, k = (1 + sqrt(3) d / s) exp(-sqrt(3) d / s),
 * d = |x - y|; s = bandwidth > 0.  The handle keeps the points: products
 * with K (cphifi_kernel_apply, and the alternating fit's A_k = K W) then
 * generate K's entries instead of reading a stored matrix.
 * cphifi_kernel_apply: Y = K X for X, Y n x r (column-major, r <= 64, memory
 * kind mem).  With points, K's tiles are generated on the fly: precision
 * CPHIFI_FP64 in FP64, CPHIFI_MIXED_FP32 in FP32 with the hardware
 * exponential (about 1e-6 relative); without points, Y = U_K (D_K o (U_K' X))
 * in FP64 from the stored eigendecomposition. */
enum cphifi_kernel_kind { CPHIFI_KERNEL_GAUSSIAN = 0, CPHIFI_KERNEL_MATERN32 = 1 };
int cphifi_kernel_create_points(cphifi_ctx* ctx, int64_t n, int32_t dim, const double* x,
                                int32_t kind, double bandwidth, int mem, cphifi_kernel** out);
int cphifi_kernel_apply(const cphifi_kernel* kern, int32_t precision, int32_t r,
                        const double* X, double* Y, int mem);
/* The eigendecomposition the kernel handle holds (Eq. eigK): UK (n x n,
 * column-major, column j = eigenvector j) and DK (n eigenvalues; ascending
 * when the library computed them), FP64, copied to memory kind `mem`.
 * Either output may be NULL. */
int cphifi_kernel_eig(const cphifi_kernel* kern, double* UK, double* DK, int mem);

/* ---- one subproblem (§4: everything that depends on the observations) ---
 * d_other     : number of other (finite) modes, >= 1.
 * other_sizes : n_m for m = 1..d_other (host array).
 * factors     : host array of d_other pointers; factor m is n_m x r,
 *               column-major, in memory kind `mem`.
 * r           : rank, 1 <= r <= 64.
 * q           : number of observations, 0 <= q < 2^31.
 * kidx        : q kernel-mode indices in [0, n).
 * oidx        : q x d_other other-mode indices, row-major (observation l's
 *               indices are oidx[l*d_other .. l*d_other + d_other - 1]),
 *               index m in [0, n_m).
 * vals        : q observed values t_l: double, or float with
 *               CPHIFI_VALS_F32.
 * flags       : CPHIFI_OBS_SORTED, CPHIFI_NEED_FP64 / CPHIFI_NEED_LOWP,
 *               CPHIFI_KEEP_OBS, CPHIFI_VALS_F32.
 * Builds on the device: the stable sort by kernel index, Zhat (Eq. zhat) in
 * the sorted order, the Gram V = Hadamard of A_m'A_m (§3), eig(V)
 * (Eq. eigV), the density gamma = q/(nM) and the preconditioner diagonal D
 * (§4.4.2).  Invalid indices or non-finite inputs give CPHIFI_E_INVALID_ARG;
 * a footprint over the context budget gives CPHIFI_E_ADMISSION. */
int cphifi_problem_create(cphifi_ctx* ctx, const cphifi_kernel* kern,
                          int32_t d_other, const int64_t* other_sizes,
                          const double* const* factors, int32_t r, int64_t q,
                          const int32_t* kidx, const int32_t* oidx,
                          const void* vals, uint32_t flags, int mem,
                          cphifi_problem** out);
int cphifi_problem_destroy(cphifi_problem* prob);
/* Device bytes the problem holds. */
size_t cphifi_problem_bytes(const cphifi_problem* prob);

/* PCG solve of Eq. unaligned-infinite-1 (§4.4).  W0 (n x r, may be NULL =
 * zero start) and W_out (n x r) are column-major in memory kind `mem`.
 * Returns CPHIFI_OK when the FP64 true relative residual is <= tol,
 * CPHIFI_E_NOT_CONVERGED at max_iter (W_out and stats still written), or
 * CPHIFI_E_BREAKDOWN. `stats` may be NULL. */
int cphifi_problem_solve(cphifi_problem* prob, const cphifi_params* params,
                         const double* W0, double* W_out, int mem,
                         cphifi_stats* stats);

/* One-shot: problem_create + problem_solve + problem_destroy.  flags as in
 * problem_create; params->precision selects the operator data built. */
int cphifi_solve(cphifi_ctx* ctx, const cphifi_kernel* kern, int32_t d_other,
                 const int64_t* other_sizes, const double* const* factors,
                 int32_t r, int64_t q, const int32_t* kidx,
                 const int32_t* oidx, const void* vals, uint32_t flags,
                 const cphifi_params* params, const double* W0, double* W_out,
                 int mem, cphifi_stats* stats);

/* ---- batches of independent solves: submit / poll / wait ------------------
 * Each kernel-mode subproblem of §4.4 (one tensor, one kernel mode, one ALS
 * sweep) is an independent PCG solve; many of them can share the GPU.  A
 * submitted request holds the arguments of cphifi_solve.  It is admitted --
 * its problem created on a stream of its own, its PCG started -- as soon as
 * fewer than `max_active` requests run and its device footprint fits the
 * context's HBM budget next to the running ones.  Pending requests are
 * considered oldest first, but one that cannot start yet is passed over by
 * smaller ones behind it: a request whose footprint (problem plus creation
 * temporaries) exceeds 1 GiB is "large", and large requests hold at most a
 * quarter of the slots (at least one), so a burst of large requests, or one
 * waiting for memory, does not hold up the small ones.  A request pending
 * for more than 50 ms is overtaken by nobody: from it on, admission is in
 * submission order until it starts.  Admitted requests advance concurrently on their own
 * streams: each PCG chunk (k_replace iterations and the true-residual check
 * of §4.4 mixed mode) is replayed from a CUDA graph captured on first use,
 * and the host only looks at a request between chunks.
 *
 * cphifi_submit   queues a request and returns its ticket at once.  The
 *                 caller keeps every buffer it names (factors, observation
 *                 lists, W0, W_out) and the kernel handle alive and unchanged
 *                 until cphifi_wait returns for that ticket.  Device-memory inputs are read
 *                 in order after the work the caller queued on the stream set
 *                 by cphifi_ctx_set_stream before the submit.  A request whose
 *                 footprint exceeds the budget even alone completes with
 *                 CPHIFI_E_ADMISSION.  Argument errors return at once.
 * cphifi_poll     advances every request without blocking.  Optional
 *                 outputs: the numbers running and queued, and up to
 *                 `done_cap` tickets (oldest first) that completed since they
 *                 were last listed and have not been waited for; cphifi_wait
 *                 on them returns at once.
 * cphifi_wait     advances all requests until the ticket completes, or until
 *                 `timeout_us` microseconds pass (negative: no limit), which
 *                 returns CPHIFI_E_TIMEOUT and leaves the request running.
 *                 On completion it writes W_out (already written when it
 *                 returns), fills `stats` (queue_ms: the wait for admission;
 *                 setup_ms: the host time of the problem's creation) and
 *                 returns the solve's status; the ticket is then released.
 * cphifi_ctx_set_slots sets max_active (1..1024, default 16).
 * Destroying the context releases requests that were never waited for. */
typedef uint64_t cphifi_ticket;
int cphifi_ctx_set_slots(cphifi_ctx* ctx, int max_active);

/* ---- launch shapes per problem size (set by an autotuner) -----------------
 * A problem of kernel size n, q observations and rank r belongs to the bucket
 * (floor(log2 n), floor(log2 max(q, 1)), r).  cphifi_ctx_set_tuning stores
 * the launch shapes for one bucket (t = NULL removes the entry); problems
 * created afterwards in that bucket -- by problem_create, solve, submit or
 * als -- use them instead of the built-in heuristics.  A field of 0 keeps the
 * heuristic value; the others are clamped to what each kernel supports.
 * Shapes change the order of floating-point sums (results stay within the
 * arithmetic's bounds) but never the results' determinism: a given context
 * and problem always give the same bits.  No counterpart in the paper. */
typedef struct cphifi_tuning {
  int32_t gds_warps_per_sm; /* gather-dot/scatter warps per SM, at most (16) */
  int32_t split32;          /* k-range splits of the FP32 n x n products    */
  int32_t split_tc;         /* ... of the tensor-core (TF32/BF16) products  */
  int32_t split_wide;       /* ... of the FP64-accurate products            */
  int32_t split64;          /* ... of the FP64 products                     */
  int32_t reserved[3];
} cphifi_tuning;
int cphifi_ctx_set_tuning(cphifi_ctx* ctx, int32_t n_log2, int32_t q_log2, int32_t r,
                          const cphifi_tuning* t);
int cphifi_submit(cphifi_ctx* ctx, const cphifi_kernel* kern, int32_t d_other,
                  const int64_t* other_sizes, const double* const* factors,
                  int32_t r, int64_t q, const int32_t* kidx,
                  const int32_t* oidx, const void* vals, uint32_t flags,
                  const cphifi_params* params, const double* W0, double* W_out,
                  int mem, cphifi_ticket* ticket);
int cphifi_poll(cphifi_ctx* ctx, int32_t* n_active, int32_t* n_pending,
                cphifi_ticket* done, int32_t done_cap, int32_t* n_done);
int cphifi_wait(cphifi_ctx* ctx, cphifi_ticket ticket, int64_t timeout_us,
                cphifi_stats* stats);

/* ---- many solves in one persistent launch ---------------------------------
 * cphifi_solve_batch solves `count` independent kernel-mode subproblems
 * (§4.4), each given as cphifi_solve's arguments, with the mixed-precision
 * PCG (params->precision must be CPHIFI_MIXED_FP32, params->gram 0; zero
 * start; one params for all items).  The problems are created first, on
 * streams of the context, without host waits (as cphifi_submit does); then
 * ONE kernel launch runs every solve.  In it each solve is a chain of phases
 * (set-up, right-hand side, restart, the five phases of a PCG iteration, the
 * four of the FP64-accurate true residual every k_replace iterations, the
 * final W = U_K Wbar), each phase a set of tiles; the blocks claim tiles
 * from a device work list (of the solves with an unclaimed tile, the one
 * that has run the most iterations, the one with the least work per
 * iteration among equals), and the block that finishes the last tile of a
 * phase takes that solve's decisions (step sizes, convergence, restart) on
 * the device and runs a tile of the next phase itself.  A solve's result is
 * the same, bit for bit, whatever else is in the batch.  The kernel's only
 * wait is that of its idle blocks; it ends with CPHIFI_E_TIMEOUT for the
 * unfinished solves if no tile finished anywhere for the context's batch
 * wait (4 seconds unless cphifi_ctx_set_batch_wait changed it).
 * items[k].W_out is n_k x r_k, column-major, in memory kind `mem` (the
 * other pointers as in cphifi_solve, memory kind `mem` too); count <= 65535.
 * stats: NULL or
 * `count` entries; solve_ms is the persistent launch's device time and
 * setup_ms the host time of all creations (the same in every entry), iter_ms
 * the device time from the launch's start to this solve's completion.
 * info (may be NULL) describes the launch.  Returns CPHIFI_OK when every
 * solve converged, else the status of the first item (in the order given)
 * that did not; argument and creation errors return before any launch and
 * name the item in cphifi_last_error.  No counterpart in the paper. */
typedef struct cphifi_batch_item {
  const cphifi_kernel* kern;
  int32_t d_other;
  int32_t r;
  const int64_t* other_sizes;
  const double* const* factors;
  int64_t q;
  const int32_t* kidx;
  const int32_t* oidx;
  const void* vals;
  uint32_t flags;     /* as in cphifi_problem_create                          */
  /* 0 in normal use.  1 holds the item back: it is created, but no block
   * ever claims a tile of it, so the launch can end only by its bounded
   * wait; the item reports CPHIFI_E_TIMEOUT (its W_out is left undefined),
   * the others their own results, and info->timed_out is 1.  This is how
   * the wait's expiry is exercised without any device fault.               */
  uint32_t hold;
  double* W_out;
} cphifi_batch_item;

typedef struct cphifi_batch_info {
  double create_ms;   /* host time of queueing every problem's creation      */
  double kernel_ms;   /* device time of the persistent launch                */
  double total_ms;    /* the whole call                                       */
  int64_t tiles;      /* tiles the launch ran                                 */
  int32_t blocks;     /* blocks of the persistent launch                      */
  int32_t timed_out;  /* 1: the launch's bounded wait expired                 */
} cphifi_batch_info;

int cphifi_solve_batch(cphifi_ctx* ctx, int32_t count, const cphifi_batch_item* items,
                       const cphifi_params* params, int mem, cphifi_stats* stats,
                       cphifi_batch_info* info);

/* cphifi_ctx_set_batch_wait: the bound of the persistent launch's idle wait,
 * in milliseconds (1 .. 600000; 4000 when never set).  The launch gives up,
 * and reports CPHIFI_E_TIMEOUT for every unfinished solve, once no tile has
 * finished anywhere for that long.  Returns CPHIFI_E_INVALID_ARG outside the
 * range. */
int cphifi_ctx_set_batch_wait(cphifi_ctx* ctx, int32_t ms);

/* ---- the steps of the path, one call each (for checking each step) ------
 * All n x r arrays are column-major in memory kind `mem`. */

/* B = T Z (sparse MTTKRP, §4) and b = vec(K B) (right-hand side of
 * Eq. unaligned-infinite-1), both n x r, FP64.  Either output may be NULL. */
int cphifi_problem_rhs(cphifi_problem* prob, double* B_out, double* b_out,
                       int mem);
/* Y = (F'F + lambda (I (x) K) + rho I) X (§4.4.1) in the operator arithmetic
 * `precision` (FP64 or one of the mixed modes); X, Y n x r FP64. */
int cphifi_problem_matvec(cphifi_problem* prob, int precision, double lambda,
                          double rho, const double* X, double* Y, int mem);
/* Y1 = Yhat1 of Eqs. vl and yhat1 for a given Xhat (n x r):
 * xbar_l = Xhat(i_l,:).Zhat(l,:), Yhat1(i,:) = sum_{i_l = i} xbar_l Zhat(l,:),
 * in FP64, double-float (FP64_EMULATED) or (mixed modes) FP32 arithmetic.
 * With precision | CPHIFI_GRAM_FORM (here and in cphifi_problem_matvec) the
 * product applies the per-index Gram blocks instead (see cphifi_params.gram):
 * FP32 blocks for the mixed modes, FP64-accurate ones otherwise. */
#define CPHIFI_GRAM_FORM 0x100
int cphifi_problem_gds(cphifi_problem* prob, int precision, const double* Xhat,
                       double* Y1, int mem);
/* The per-index Gram blocks C_i = sum over l with i_l = i of
 * Zhat(l,:)'Zhat(l,:) (the r x r diagonal blocks of H in
 * F'F = (I (x) K) H (I (x) K), §4.4.1), as the solver holds them: FP32 (mixed
 * modes, returned widened to FP64) or FP64-accurate (FP64, FP64_EMULATED).
 * C: n r^2 doubles, C[(i r + j) r + k] = C_i(j, k), in memory kind mem.
 * Builds the blocks if the problem has none yet. */
int cphifi_problem_grams(cphifi_problem* prob, int precision, double* C, int mem);
/* Y = M^{-1} X for the preconditioner of Eq. precon, applied as Eq. fx. */
int cphifi_problem_precond(cphifi_problem* prob, double lambda, double rho,
                           const double* X, double* Y, int mem);
/* V = Z'Z (r x r), its eigenvalues DV (r) and eigenvectors UV (r x r,
 * column-major) as computed on the device (Eq. eigV); any may be NULL.
 * Host memory only. */
int cphifi_problem_gram(cphifi_problem* prob, double* V, double* DV,
                        double* UV);
/* The sorted observation order: perm[s] = original index of the s-th
 * observation after the stable sort by kernel index, and row_ptr (n+1) with
 * observations of kernel index i at sorted positions [row_ptr[i],
 * row_ptr[i+1]).  Host memory only; either may be NULL. */
int cphifi_problem_order(cphifi_problem* prob, int32_t* perm,
                         int64_t* row_ptr);

/* ---- the alternating fit around the kernel-mode solve (§2) ----------------
 * The CP-HIFI model (§2) is a rank-r CP tensor whose kernel-mode factor is
 * A_k = K W and whose other (finite) modes have plain factors A_m; it is fit
 * by alternating over the modes (§2, Eq. cp-hifi-subproblem).  The kernel
 * mode is the PCG solve above; a finite mode has no regulariser (R_m = 0,
 * §2), so its update is the CP-ALS step for incomplete data: with
 * z_l = A_k(i_l,:) o prod_{m' != m} A_m'(i_m'^l,:), row i of A_m solves the
 * r x r normal equations G_i a = h_i, G_i = sum z_l z_l', h_i = sum t_l z_l
 * over the observations with i_m^l = i (FP64 sums, Cholesky).  The paper
 * only cites this step as known; this library adds 1e-12 trace(G_i) to the
 * diagonal of rows with fewer than r observations and leaves rows without
 * observations (or whose G_i is not positive definite after that) unchanged.
 * These calls need a problem created with CPHIFI_KEEP_OBS.
 *
 * cphifi_problem_set_factors: replaces the finite factors (n_m x r,
 *   column-major, memory kind mem) and rebuilds what depends on them (Zhat,
 *   the MTTKRP B, V, eig(V)); the observation order is kept.
 * cphifi_problem_update_factor: the CP-ALS update of finite mode m for the
 *   kernel weights W (n x r): A_k = U_K (D_K o (U_K' W)) in FP64, the
 *   normal equations, Cholesky.  The new factor replaces the problem's
 *   (and is copied to A_out, n_m x r, when A_out is not NULL); the data that
 *   depend on it are rebuilt before the next solve.
 * cphifi_problem_fit: for the model (K W, the problem's factors), the sums
 *   sum_l (t_l - m_l)^2 and sum_l t_l^2 in FP64 (either output may be NULL).
 * cphifi_als: the alternating fit.  Creates a problem (CPHIFI_KEEP_OBS
 *   added to flags), then per sweep: the kernel-mode PCG solve (params;
 *   warm started from the previous W, or from W_io when `warm` is set),
 *   the finite modes in order, and the relative fit error
 *   ||t - m|| / ||t|| into err_out[sweep] (err_out holds `sweeps` values).
 *   Stops after `sweeps` sweeps or when the error changes by less than
 *   als_tol (§5: tolerance on the change in the ALS error).  factors_io
 *   (d_other pointers, each n_m x r) are read as the start and overwritten
 *   with the fitted factors; W_io (n x r) receives the fitted weights.  All
 *   in memory kind mem.  *sweeps_done (may be NULL) gets the number of
 *   sweeps run; `stats` (may be NULL) the last kernel-mode solve's stats. */
int cphifi_problem_set_factors(cphifi_problem* prob, const double* const* factors, int mem);
int cphifi_problem_update_factor(cphifi_problem* prob, int32_t mode, const double* W,
                                 double* A_out, int mem);
int cphifi_problem_fit(cphifi_problem* prob, const double* W, int mem, double* res2,
                       double* t2);
int cphifi_als(cphifi_ctx* ctx, const cphifi_kernel* kern, int32_t d_other,
               const int64_t* other_sizes, double* const* factors_io, int32_t r,
               int64_t q, const int32_t* kidx, const int32_t* oidx, const void* vals,
               uint32_t flags, const cphifi_params* params, int32_t sweeps, double als_tol,
               int32_t warm, double* W_io, double* err_out, int32_t* sweeps_done, int mem,
               cphifi_stats* stats);

/* ---- allocation-free entry point -----------------------------------------
 * cphifi_gds_noalloc: the gather-dot/scatter product of the solver, FP64,
 * without allocating device memory.  There is no counterpart in the paper:
 * it exists for callers that cannot call cudaMalloc (for example a real-time
 * host loop that may not take the allocator's locks or wait for its implicit
 * device synchronisation, or a runtime that owns all device memory and lets
 * no library take more).  The caller passes inputs and outputs; the working
 * memory comes from a fixed array of about 10.7 MB compiled into the
 * library, which every GPU that loads the library keeps until the process
 * exits.
 *   n, r     : kernel-mode size in [1, 16384] and rank in [1, 64]; larger
 *              sizes return CPHIFI_E_INVALID_ARG with *err_msg naming the limit.
 *   q        : number of observations, in [0, 2^31).
 *   row_ptr  : device, n+1 int64: observations of kernel index i occupy
 *              sorted positions [row_ptr[i], row_ptr[i+1]).  It must be a CSR
 *              of q entries: row_ptr[0] = 0, non-decreasing, row_ptr[n] = q.
 *              This is checked on the device: otherwise no memory but Y1 is
 *              written and Y1 is filled with NaN (the call itself has already
 *              returned CPHIFI_OK, since the check runs on the stream).
 *   zhat     : device FP64, Zhat in that sorted order, column-major q x r with
 *              leading dimension ldz >= q.
 *   Xhat     : device FP64 n x r column-major (leading dimension n).
 *   Y1       : device FP64 n x r column-major: Y1(i,:) = sum over the
 *              observations l of index i of (Xhat(i,:).Zhat(l,:)) Zhat(l,:).
 *   stream   : cudaStream_t the work is queued on (NULL = legacy default).
 *   err_msg  : optional; set to a static string describing the outcome.
 * Runs on the calling thread's current device and returns once the work is
 * queued (asynchronous: synchronise `stream` before reading Y1).  The first
 * call on a device looks up the device address of the scratch array (a
 * failed lookup is retried by the next call); make that first call before
 * any stream capture.  Every call on a device shares the scratch array, and
 * each call clears what must start at zero, so calls that overlap on the GPU
 * (other streams or host threads) race: serialise them on one stream.
 * Returns CPHIFI_OK, CPHIFI_E_INVALID_ARG or CPHIFI_E_DEVICE. */
int cphifi_gds_noalloc(int32_t n, int32_t r, int64_t q, const int64_t* row_ptr,
                       const double* zhat, int64_t ldz, const double* Xhat,
                       double* Y1, void* stream, const char** err_msg);

#ifdef __cplusplus
}
#endif
#endif /* CPHIFI_H */
