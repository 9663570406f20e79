/*
 * nmf.h -- C ABI of the GB300 (sm_103a) streaming-NMF library.
 *
 * The library implements the hot path of the two-stage method of Gu, Du and
 * Billinge, "A fast two-stage algorithm for non-negative matrix factorization
 * in streaming data" (arXiv 2101.08431): the stage-1 ANLS sweep for
 *
 *     min 1/2 ||X Y - M||_F^2   s.t.  X >= 0, Y >= 0            (eq. "prob", Sec. 1)
 *
 * with M (n x m) whose columns are time instants that arrive progressively
 * (Sec. 1).  Each sweep solves every column of Y and then every row of X as an
 * independent nonnegative least-squares problem (eq. "qp", Sec. 2) with the
 * Lawson-Hanson active-set method warm-started from the previous solution
 * and its passive set (Sec. 2).
 *
 * Conventions for every entry point:
 *   - Layouts: M and appended columns are column-major (element (i, j) at
 *     i + ld*j); X is n x k row-major (X[i*k + a], the vector x = vec(X^T) of
 *     Sec. 3.1); Y is k x m column-major (Y[a + k*j], y = vec(Y)); passive-set
 *     masks are one uint32 per column of Y / row of X, bit a set when
 *     component a is positive.
 *   - Pointers are borrowed for the duration of the call only; data are
 *     copied into library-owned device memory.  `on_device` = 1 means the
 *     pointer is CUDA device memory, 0 means host memory (pinned host memory
 *     gives asynchronous copies).  Output buffers belong to the caller.
 *   - Streams: all device work of a handle is ordered on the stream given in
 *     its nmf_config (NULL: the library creates one).  Calls that return data
 *     to the host (nmf_get_factors, nmf_objective_kkt, nmf_sweep when it
 *     fills stats) synchronise that stream.
 *   - Errors: every call returns an nmf_status; nothing aborts or throws
 *     across the ABI.  After NMF_ECUDA or NMF_ETIMEOUT the handle is poisoned
 *     (every later call returns the same status) until nmf_destroy.
 *     nmf_last_error gives a one-line explanation of the last failure.
 *   - Threading: a handle is used by one thread at a time; distinct handles
 *     are independent.
 */
#ifndef NMF_GB300_H
#define NMF_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nmf_handle nmf_handle;

typedef enum {
    NMF_OK = 0,
    NMF_EINVAL = 1,      /* bad argument or unsupported size                 */
    NMF_ENOMEM = 2,      /* device or host allocation failed                 */
    NMF_ECUDA = 3,       /* CUDA runtime error (handle poisoned)             */
    NMF_ENOTCONV = 4,    /* iteration cap reached before the stopping test   */
    NMF_ETIMEOUT = 5,    /* a bounded device wait gave up (handle poisoned)  */
    NMF_ECAPACITY = 6,   /* request exceeds the handle's capacity            */
    NMF_ENUMERIC = 7,    /* NaN or Inf in the data or the iterates           */
    NMF_ESTATE = 8       /* call out of order (e.g. sweep before factors)    */
} nmf_status;

typedef enum {
    NMF_PREC_FP64 = 0,   /* M stored and contracted in FP64                  */
    NMF_PREC_MIXED = 1   /* M stored FP32; FP32 passes, then compensated
                            (double-float) refinement passes; NNLS, Grams
                            and KKT in FP64                                  */
} nmf_precision;

enum { NMF_DTYPE_F64 = 0, NMF_DTYPE_F32 = 1 };
/* Warm start of the column solves (Sec. 2): cold; from the column's own
 * previous-sweep solution (all columns in parallel); or the paper's chain,
 * column j from column j - 1's new solution, one column after another over
 * the whole window (one CTA; k <= 8 -- rank 16 solves from the previous
 * sweep) -- the sequential form whose active-set savings Sec. 2 argues for. */
enum { NMF_WARM_COLD = 0, NMF_WARM_PREV = 1, NMF_WARM_CHAIN = 2 };

typedef struct {
    int64_t n;               /* rows of M (distance grid)                     */
    int64_t m_capacity;      /* resident time columns (ring buffer capacity)  */
    int32_t k;               /* rank, 1..8 or 16 (see nmf_create)             */
    int32_t prec;            /* nmf_precision                                 */
    double stol;             /* eps_STOL of the Sec. 4 relative step test;
                                <= 0 disables                                 */
    double kkt_target;       /* stop when the relative KKT error <= target;
                                <= 0 disables                                 */
    double mixed_switch;     /* MIXED: move to the refinement passes once the
                                relative KKT error <= this (or stalls)       */
    int32_t max_sweeps;      /* cap for nmf_sweep(h, 0, ...)                  */
    int32_t warm_start;      /* NMF_WARM_COLD, NMF_WARM_PREV or NMF_WARM_CHAIN */
    void *cuda_stream;       /* cudaStream_t, or NULL                         */
    double kkt_abs_target;   /* also stop when the absolute KKT error E (Sec.
                                5.1's stopping rule, eps_TOL) <= this; <= 0
                                disables                                      */
} nmf_config;

typedef struct {
    int32_t sweeps;          /* sweeps run by this call                        */
    int32_t iter;            /* index of the current iterate                   */
    int32_t converged;       /* 1 rel-KKT target met, 2 step test met, 0 not   */
    int32_t fp64_sweeps;     /* sweeps of this call in the refinement phase:
                                FP64-accurate contractions (FP64, compensated
                                or incremental M pass)                        */
    double f;                /* 1/2 ||XY - M||^2 of the last measured iterate  */
    double kkt_abs;          /* E(x, y, r, s; 0) with r = max(graX,0),
                                s = max(graY,0) (Sec. 5.1), 2-norms            */
    double kkt_rel;          /* kkt_abs terms scaled (see nmf_objective_kkt)   */
    double step_rel;         /* ||Δ(x,y)|| / (1 + ||(x,y)||) (Sec. 4)          */
    int64_t changed_cols;    /* columns whose passive set changed (last sweep) */
    int64_t changed_rows;    /* rows whose passive set changed (last sweep)    */
    int64_t nnls_notconv;    /* NNLS solves that hit their iteration cap       */
    int32_t measured_iter;   /* iterate the f / KKT figures belong to          */
    int32_t entering_steps;  /* Lawson-Hanson entering steps of the column
                                solves of the sweep that measured the record  */
} nmf_stats;

/* Defaults: stol 0, kkt_target 1e-8, kkt_abs_target 0, mixed_switch 1e-6,
 * max_sweeps 100000, warm_start NMF_WARM_PREV, prec NMF_PREC_MIXED. */
void nmf_config_init(nmf_config *cfg);

/* Create a handle for one problem of n rows, rank k and up to m_capacity
 * resident columns (Sec. 1's streaming setting).  Allocates all device
 * memory up front; no allocation happens in later calls except
 * nmf_append_columns' staging of host data and the work memory of the
 * stage-2 calls (nmf_ipm, nmf_ipm_direction) and of the first shard call.  Errors: NMF_EINVAL for n < 1,
 * k outside 1..8 and 16, m_capacity < 1 or n beyond the kernels' row limit
 * (16384 rows FP32, 8192 FP64); NMF_ENOMEM; NMF_ECUDA.
 * Ranks: the passive-set masks would hold k <= 32, but the kernels are built
 * for k = 1..8 (subset tables of inv(G_PP) for all 2^k passive sets, lanes of
 * a warp per problem) and k = 16 (one 16-lane group per problem, the
 * tensor-core contractions of the mixed form); other ranks are rejected.
 * Rank 16 with NMF_PREC_MIXED: the FP32-class pass runs on the tensor cores
 * (split-BF16 contractions, about 1e-5 relative in B and P, in two streaming
 * launches with the FP32 column solves between them; row solves predicted in
 * FP32, refined and checked in FP64).
 * Where n is beyond the rows of the cluster-fused FP64-class kernels at rank
 * 16 (n above about 3840), the refinement runs the rank-16 reference pass
 * (compensated FP32 "double-float" B = X^T M and P = M Y^T, FP64 solves;
 * pass modes 1 and 2, the recording sweep of mode 3, the priming pass and
 * nmf_objective_kkt) and the incremental pass (tensor-core contractions of
 * the change of X and Y since the reference sweep added to its FP64
 * contractions; mode 3).  Such a handle also holds M with its first 128
 * columns repeated after the ring (tensor copies never wrap). */
nmf_status nmf_create(const nmf_config *cfg, nmf_handle **out);

/* The configuration the handle was created with (its cuda_stream field is
 * the stream the handle's work is ordered on).  NMF_EINVAL for NULL. */
nmf_status nmf_get_config(const nmf_handle *h, nmf_config *out);

/* Free every resource of the handle (NULL is accepted). */
nmf_status nmf_destroy(nmf_handle *h);

/* Append ncols time columns (n x ncols, column-major, leading dimension ld,
 * dtype NMF_DTYPE_F32/F64) to the resident window (Sec. 1: data arrive by
 * columns).  When the window would exceed m_capacity the oldest columns are
 * evicted.  A new column's y is seeded with the last resident column's y and
 * passive set (the continuity of Sec. 2's warm start).  FP64 input is
 * rounded to FP32 in NMF_PREC_MIXED handles.  Returns NMF_ENUMERIC (data
 * stored, handle usable) if a value is NaN or Inf; NMF_EINVAL for ld < n. */
nmf_status nmf_append_columns(nmf_handle *h, const void *cols, int64_t ncols, int64_t ld,
                              int32_t dtype, int32_t on_device);

/* Number of resident columns m. */
int64_t nmf_num_columns(const nmf_handle *h);

/* Set the iterate: X (n x k row-major) and Y (k x m column-major for the m
 * resident columns, FP64).  Negative entries are set to 0.  Runs one priming
 * pass over M so that the first sweep can report the iterate's KKT error.
 * NMF_ESTATE if no column is resident. */
nmf_status nmf_set_factors(nmf_handle *h, const double *X, const double *Y, int32_t on_device);

/* Copy the current iterate out (X n x k, Y k x m, masks may be NULL).
 * Synchronises the stream. */
nmf_status nmf_get_factors(nmf_handle *h, double *X, double *Y, uint32_t *xmask, uint32_t *ymask,
                           int32_t on_device);

/* Run ANLS sweeps (Alg. "anls", Sec. 2; Y-update then X-update).  nsweeps > 0
 * runs that many (fewer if a stopping test holds); nsweeps == 0 runs until
 * the relative KKT target or the step tolerance is met, or max_sweeps
 * (NMF_ENOTCONV).  The KKT error of iterate t is measured during sweep t from
 * the Grams (no second read of M); when the target holds, the handle keeps
 * iterate t.  stats (may be NULL) describes the last measured iterate; a
 * non-NULL stats synchronises the stream. */
nmf_status nmf_sweep(nmf_handle *h, int32_t nsweeps, nmf_stats *stats);

/* NMF_PREC_MIXED handles: force the arithmetic of the following M passes
 * (0 = FP32 contraction, 1 = FP64-accumulated contraction of the FP32 M,
 * 2 = compensated FP32 (double-float) contraction of the FP32 M, about 44
 * significant bits; 3 = incremental: every chunk of up to 32 sweeps starts
 * with a compensated sweep that records its contractions B_ref = X_t^T M and
 * P_ref = M Y_{t+1}^T as references, and its other sweeps form
 * B = B_ref + (X - X_t)^T M and P = P_ref + M (Y - Y_{t+1})^T with the change
 * terms contracted in FP32 -- their rounding is 2^-24 of the change, so
 * near convergence the sweep is as accurate as the compensated one at the
 * cost of an FP32 pass; -1 = automatic: FP32 until the relative KKT error
 * reaches mixed_switch or stalls, then incremental (compensated where the
 * incremental pass has no launch plan)).  NMF_PREC_FP64 handles ignore it.
 * At rank 16, mode 0 is the tensor-core pass (see nmf_create).
 * NMF_EINVAL for any other mode. */
nmf_status nmf_set_pass_mode(nmf_handle *h, int32_t mode);

/* Objective and KKT error of the current iterate from one read-only,
 * FP64-accumulated pass over M plus the Grams: f = 1/2||XY - M||^2,
 * kkt_abs = max{||(min(graX,0), min(graY,0))||, ||(r o X, s o Y)||} (eq.
 * "error" with mu = 0 and the duals of Sec. 5.1), kkt_rel = max{ first term /
 * s_g, second term / (s_g max(max X, max Y)) } with s_g = ||M Y^T||_F +
 * ||X^T M||_F.  Any output pointer may be NULL.  Synchronises the stream. */
nmf_status nmf_objective_kkt(nmf_handle *h, double *f, double *kkt_abs, double *kkt_rel);

/* Static description of a status code. */
const char *nmf_status_string(nmf_status s);

/* Detail of the handle's last failure ("" if none). */
const char *nmf_last_error(const nmf_handle *h);

/* Number of kernel launches the handle has issued so far (for accounting). */
int64_t nmf_launch_count(const nmf_handle *h);

/* Per-kernel device timing: with on = 1 every later sweep brackets its M
 * pass and its row pass with CUDA events on the handle's stream; on = 0
 * stops.  Each call resets the accumulated figures. */
nmf_status nmf_set_timing(nmf_handle *h, int32_t on);

/* Accumulated device time (ms) and launch counts of the M pass (ypass) and
 * of the row pass (xpass) since nmf_set_timing(h, 1).  Synchronises the
 * stream.  Any output pointer may be NULL. */
nmf_status nmf_get_timing(nmf_handle *h, double *ypass_ms, int64_t *ypass_launches,
                          double *xpass_ms, int64_t *xpass_launches);

/* Persistence of a stream's state (the streaming setting of Sec. 1 keeps a
 * problem resident for as long as its columns keep arriving; these calls let
 * that state outlive the process).  nmf_save writes to the file at path: the
 * configuration (without its stream), the resident window of M in logical
 * column order, the current iterate X, Y with its passive sets and Gram G
 * (and, k <= 8, G's subset table), the device control block (iterate index,
 * statistics, KKT terms of the iterate, ||M||^2) and the mixed schedule's
 * state.  It synchronises the handle's stream and leaves the handle as it
 * was.  nmf_load creates a new handle on cuda_stream (NULL: the library
 * creates one) holding that state, with the window in the ring's first
 * columns; sweeps of the loaded handle give bitwise the results the saved
 * handle would give (the sweep's partitions follow logical column order).
 * The file is in the byte order of the machine that wrote it (little-endian
 * on the x86-64 and Arm hosts this library builds for) and is specific to
 * this library version: nmf_load rejects a file whose header, sizes or length
 * do not match (NMF_EINVAL, before any device allocation).  Errors: NMF_EINVAL
 * for NULL arguments or a path that cannot be opened, read or written; the
 * errors of nmf_create; NMF_ECUDA. */
nmf_status nmf_save(nmf_handle *h, const char *path);
nmf_status nmf_load(const char *path, void *cuda_stream, nmf_handle **out);

/* Multi-GPU: the time columns sharded across ranks (one process, GPU and
 * handle per rank; each handle holds its own columns, appended as usual, and
 * the same X).  In Alg. "anls" (Sec. 2) the Y half solves every column on its
 * own, and the X half needs only P = M Y^T and H = Y Y^T summed over all
 * columns, so a sweep is:
 *   1. nmf_shard_y_half on every rank: the M pass over the rank's columns
 *      (new Y, passive sets) and the rank's P (n x k, row-major), H (k x k),
 *      Y-half KKT terms and ||M||^2, written to sum_buf
 *      (nmf_shard_buffer_len(n, k) doubles) and the largest y to max_buf
 *      (1 double);
 *   2. the caller's collective: sum_buf summed over the ranks, max_buf its
 *      maximum (e.g. two NCCL or gloo all-reduces) -- the one exchange of the
 *      sweep, n k + k^2 + 11 doubles;
 *   3. nmf_shard_x_half on every rank with the reduced buffers: the row pass
 *      (the same X on every rank, as all-reduce results are the same on every
 *      rank), G = X^T X, and the statistics of the incoming iterate over the
 *      whole problem (stats may be NULL; filling it synchronises; the first
 *      sweep after nmf_set_factors reports its incoming iterate unmeasured,
 *      kkt_rel = -1, as the priming pass saw only the rank's columns).
 * Pass: the FP64 form's pass; for NMF_PREC_MIXED handles pass mode 0 (FP32),
 * 1 (FP64-accumulated), else the compensated pass.  Buffers are host memory
 * (on_device 0; the calls then synchronise the stream) or device memory
 * (on_device 1).  The stopping tests apply to the whole problem
 * (stats.converged).  Errors: NMF_EINVAL for NULL pointers, NMF_ESTATE for a
 * Y half before factors are set, two Y halves in a row or an X half without
 * one. */
int64_t nmf_shard_buffer_len(int64_t n, int32_t k);
nmf_status nmf_shard_y_half(nmf_handle *h, double *sum_buf, double *max_buf, int32_t on_device);
nmf_status nmf_shard_x_half(nmf_handle *h, const double *sum_buf, const double *max_buf, int32_t on_device,
                            nmf_stats *stats);

/* Stage 2 of the two-stage method (Alg. "alg:fast", Sec. 3-4) on the GPU, in
 * FP64, from the handle's current iterate (its resident window): the
 * transition of Sec. 4 (eqs. "upxy", "rho0", "rs", "mu", "rho" with
 * rho = eps_tol), then the outer loop on mu with the inner Newton loop of the
 * primal-dual interior point method -- fraction to the boundary (tau = 0.9),
 * Armijo backtracking on the barrier merit function (eq. "eqn:armijo",
 * eta = 0.5, at most 60 halvings), the predictor-based sigma (eqs.
 * "eqn:muaff", "eqn:mu") and the switch to the full Hessian at
 * sigma <= 0.01 when it gives a descent direction -- until the KKT error
 * E(.;0) <= eps_tol or max_newton Newton steps.  Each direction is formed as
 * in Sec. 3.2 (block Cholesky of R1, W = Cb P^-1, the mk x mk Schur matrix
 * and its dense Cholesky).  The result becomes the handle's iterate (primed as
 * by nmf_set_factors).  stats (NULL or 7 doubles): E(.;0) at exit, f, Newton
 * steps, outer steps, final mu, steps that used the full Hessian, Armijo
 * failures.  Work memory is allocated for the call: 8 (m k (n k + m k) +
 * n k^2 + ...) bytes; NMF_ECAPACITY when m k > 4096 or n k m k > 2^27.
 * Returns NMF_ENOTCONV at the Newton cap (for n != m the printed method can
 * drift along the scaling orbit of the factorization and end there),
 * NMF_ENUMERIC if a factorisation is not positive definite, NMF_ESTATE before
 * factors are set.
 * nmf_ipm_direction: one direction of eq. "eqn:equation" at the handle's
 * iterate for duals r (n x k, like X) and s (k x m, like Y), barrier mu >= 0,
 * regularisation rho >= 0, full = 1 for the full Hessian blocks C (else the
 * Gauss-Newton blocks): dx, dy, dr, ds in the layouts of X, Y, X, Y. */
nmf_status nmf_ipm(nmf_handle *h, double eps_tol, int32_t max_newton, double *stats);
nmf_status nmf_ipm_direction(nmf_handle *h, const double *r, const double *s, double mu, double rho,
                             int32_t full, double *dx, double *dy, double *dr, double *ds, int32_t on_device);

/* The accumulated device time (ms) of the M passes and of the row passes
 * of one pass variant since nmf_set_timing(h, 1), and how many sweeps ran
 * it: pass 0 FP32, 1 FP64-accumulated, 2 compensated, 3 incremental (pass
 * modes 0..3 of the mixed form), 4 the FP64 form's pass.  Synchronises the
 * stream.  Any output pointer may be NULL; NMF_EINVAL for another pass. */
nmf_status nmf_get_pass_timing(nmf_handle *h, int32_t pass, double *ypass_ms, double *xpass_ms,
                               int64_t *sweeps);

/* One ANLS sweep that allocates no memory at all.
 *
 * The paper has no counterpart: this is a deployment variant of nmf_sweep for
 * callers that cannot allocate device memory where they run the sweep -- a
 * latency-critical loop that must never block on cudaMalloc (which can
 * synchronise the device and take milliseconds), a plug-in whose host
 * framework has reserved all device memory for its own pool, or code that
 * is allowed to allocate only during start-up.  It needs no handle and calls
 * no allocating routine.
 *
 *   M          device, n x m FP32, column-major, leading dimension ldm equal to
 *              n rounded up to a multiple of 32; rows n..ldm-1 must hold finite
 *              values (zeros, say);
 *   X, Y       device FP64: X n x k row-major, Y k x m column-major; on entry the
 *              iterate (entries >= 0), on exit the next iterate: one sweep,
 *              Y-update then X-update, with the FP64-accumulated M pass;
 *   stats_dev  NULL or a device buffer of 16 doubles that receives the record of
 *              the incoming iterate (index 1: f, 2: KKT error, 3: relative KKT)
 *              and, at index 15, the sweep's device error bits: 0 when the sweep
 *              completed, bit 0 (1) when a bounded device wait gave up, bit 1 (2)
 *              when a non-finite value was met.  With any bit set, X and Y are
 *              left holding the incoming iterate.  Pass a record to learn of
 *              these errors: the call returns before the device work runs;
 *   cuda_stream  the stream the work is ordered on (NULL: the default stream);
 *              the call returns once the work is enqueued.
 * Alignment: M must be 16-byte aligned (the M pass stages column segments with
 * bulk copies), X, Y and stats_dev 8-byte aligned; otherwise NMF_EINVAL, before
 * any device work.
 * Limits: n <= 2048, m <= 4096, 1 <= k <= 8; larger sizes return NMF_ECAPACITY,
 * a wrong ldm or a NULL pointer NMF_EINVAL.
 * Working memory: one 5 MiB __device__ array compiled into the library, which
 * every GPU that loads the library holds until the process exits.  All calls
 * share it and it keeps the last call's contents (each call re-initialises what
 * must start at zero), so calls whose work overlaps on the GPU -- on different
 * streams or from different threads -- race on it; serialise them.
 * Set-up: the first call on each device looks up the array's device address
 * with that device current; make that first call before any stream capture
 * on the device.  With CUDA's lazy module loading (the default), that first
 * call is also when the driver loads the library's kernels and places the
 * array in device memory -- an allocation by the driver -- so make it at
 * start-up, while device memory is still free, or set
 * CUDA_MODULE_LOADING=EAGER so that the array is placed when the CUDA context
 * is created. */
nmf_status nmf_sweep_noalloc(const float *M, int64_t n, int64_t m, int64_t ldm, int32_t k,
                             double *X, double *Y, double *stats_dev, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Batched form: many independent problems of uneven n, m and k, each the
 * problem of Sec. 1 with its own stopping test, swept together.  The paper
 * solves one problem at a time; batching is a deployment form of the same
 * sweep (every problem's iterates are those nmf_sweep would produce for the
 * same partition of its columns into groups).
 *
 * Execution: problems are grouped into classes by (k, cluster size); each
 * class runs one persistent launch whose clusters claim work items in list
 * order -- for every sweep, the M-pass items (problem, column group) of every
 * problem, then its row-pass items (problem, group of row blocks) -- with
 * per-problem dependency counters and bounded waits.  The classes run
 * concurrently on forked streams, and one replay of 16 sweeps is captured in
 * a CUDA graph.  The mixed-precision schedule runs on the device per problem:
 * FP32 passes until the relative KKT error reaches mixed_switch or has not
 * improved by 2% over 256 sweeps, then compensated (double-float) passes; a
 * problem stops at its own kkt_target / stol and drops out of later items.
 * Results do not depend on which other problems share the batch.
 * ------------------------------------------------------------------------ */
typedef struct nmf_batch nmf_batch;

/* Create a batch of nprob problems, problem j configured by cfgs[j] (prec
 * must be NMF_PREC_MIXED; the cuda_stream fields are ignored: every problem's
 * work is ordered on the batch's stream, cuda_stream here, NULL: the library
 * creates one).  Allocates each problem's device memory as nmf_create does.
 * Returns NMF_EINVAL for nprob < 1 or an unsupported configuration. */
nmf_status nmf_batch_create(const nmf_config *cfgs, int32_t nprob, void *cuda_stream, nmf_batch **out);

/* Release the batch and every problem in it (synchronises its stream). */
nmf_status nmf_batch_destroy(nmf_batch *b);

/* Number of problems; the handle of problem j (owned by the batch: use it
 * for read-only calls such as nmf_objective_kkt, never nmf_destroy). */
int32_t nmf_batch_size(const nmf_batch *b);
nmf_handle *nmf_batch_problem(nmf_batch *b, int32_t j);

/* Per-problem data, with the arguments and errors of nmf_append_columns,
 * nmf_set_factors and nmf_get_factors for problem j (0 <= j < nprob). */
nmf_status nmf_batch_append_columns(nmf_batch *b, int32_t j, const void *cols, int64_t ncols, int64_t ld,
                                    int32_t dtype, int32_t on_device);
nmf_status nmf_batch_set_factors(nmf_batch *b, int32_t j, const double *X, const double *Y,
                                 int32_t on_device);
nmf_status nmf_batch_get_factors(nmf_batch *b, int32_t j, double *X, double *Y, uint32_t *xmask,
                                 uint32_t *ymask, int32_t on_device);

/* Pass mode of every problem: -1 the device schedule above (default), 0 FP32
 * passes only, 2 compensated passes only.  Fixed modes stop on the targets
 * at every sweep.  Other values: NMF_EINVAL. */
nmf_status nmf_batch_set_pass_mode(nmf_batch *b, int32_t mode);

/* Schedule of the persistent launches: columns per M-pass item (the column
 * groups of each problem, so also the number of partials its row pass
 * reduces) and the largest number of TMA stages of the M pass (1..8).  The
 * partition of a problem's columns depends on cols_per_item, so results
 * agree across schedules to rounding only. */
nmf_status nmf_batch_set_schedule(nmf_batch *b, int32_t cols_per_item, int32_t stage_cap);

/* Sweep every problem that has factors and columns: max_sweeps > 0 sweeps at
 * most (fewer when every problem stops), 0: until every problem stops,
 * capped by the largest max_sweeps of the configurations (NMF_ENOTCONV when
 * the cap is reached first).  stats: NULL or nprob records, record j as
 * nmf_sweep would fill it for problem j (fp64_sweeps counts compensated
 * sweeps).  sweeps_run: NULL or the number of batch sweeps launched.
 * Synchronises the batch's stream after every 16 sweeps. */
nmf_status nmf_batch_sweep(nmf_batch *b, int32_t max_sweeps, nmf_stats *stats, int32_t *sweeps_run);

/* Autotuner: times every candidate schedule (cols_per_item in {16, 32, 64,
 * 128, 256} x stage_cap in {2, 8}) over trial_sweeps FP32-pass sweeps of the
 * batch as it stands and keeps the fastest; the tuning sweeps are ordinary
 * sweeps of the iteration (the problems advance).  Outputs (NULL allowed):
 * the chosen schedule and its time per batch sweep in ms. */
nmf_status nmf_batch_autotune(nmf_batch *b, int32_t trial_sweeps, int32_t *cols_per_item, int32_t *stage_cap,
                              double *best_ms_per_sweep);

/* Self-test of the bounded device wait used by the batched form's dependency
 * counters: one kernel waits, with a limit of `polls` polls (~256 ns each,
 * 1..2^24), on a counter that nothing increments.  Returns NMF_ETIMEOUT when
 * the wait gave up and reported it through the control block (the expected
 * outcome), NMF_OK if the wait ended otherwise, NMF_EINVAL for a bad limit.
 * The paper has no counterpart; no kernel of the library spins unbounded. */
nmf_status nmf_selftest_bounded_wait(int64_t polls, void *cuda_stream);

/* Self-test of the bounded wait of the rank-16 tensor-core M pass: one kernel
 * waits, through that pass's wait function, on an mbarrier nothing arrives
 * on, with a wall-time limit of limit_ms (1..10000; the pass itself uses
 * 2000).  Returns NMF_ETIMEOUT when the wait gave up and raised the pass's
 * abort flag (the expected outcome), NMF_OK if it ended otherwise, NMF_EINVAL
 * for a bad limit.  The paper has no counterpart. */
nmf_status nmf_selftest_tc16_wait(int64_t limit_ms, void *cuda_stream);

/* Measured FMA throughput of the current device, the denominators of the ALU
 * rooflines (the FP64 form's M pass, the SIMT passes): out[0] = FP64, out[1]
 * = FP32, in TFLOP/s (2 flops per FMA), each from one launch of independent
 * FMA chains on every SM (after an untimed one) timed with CUDA events on
 * cuda_stream (NULL: the legacy default stream).  out: 2 doubles of host
 * memory, written on NMF_OK.  Allocates a 2 KB sink and two events and frees
 * them.  Returns NMF_EINVAL for a NULL out, NMF_ECUDA on a CUDA error.  The
 * paper has no counterpart. */
nmf_status nmf_measure_fma_peaks(double *out, void *cuda_stream);

/* Kernel launches issued by the batch (graph replays count their launches). */
int64_t nmf_batch_launch_count(const nmf_batch *b);
const char *nmf_batch_last_error(const nmf_batch *b);

/* ------------------------------------------------------------------------
 * Streaming server: many streams whose time columns arrive in chunks (the
 * streaming setting of Sec. 1), served by a worker thread of the library.
 * Every admitted stream's ring of columns (capacity m_capacity; older
 * columns are evicted), X, Y and passive sets stay resident on the device;
 * each chunk is appended with its columns warm-started from the stream's
 * last column (y and passive set) and the stream's current X.  Rounds:
 * append every chunk that has arrived, then run sweeps_per_round batched
 * sweeps (the batched form above) over every stream with chunks in flight
 * -- continuous batching: chunks that arrive during a round join at the
 * next round, and the work of all streams of a round overlaps in the same
 * launches.  A chunk completes, together with the stream's other chunks in
 * flight, when the stream's relative KKT error reaches kkt_target, or after
 * max_sweeps_per_chunk sweeps.  Streams are admitted in the order they were
 * opened while their device footprint fits hbm_budget_bytes and at most
 * max_streams are resident; closing a stream (after its chunks complete)
 * frees its memory for the next one.  A stream's results do not depend on
 * the other streams being served (the batched form's property), for the
 * same sequence of its own chunks and rounds.
 * ------------------------------------------------------------------------ */
typedef struct nmf_server nmf_server;

typedef struct {
    int64_t hbm_budget_bytes;     /* device bytes the streams may hold; 0: 90% of free memory */
    int32_t max_streams;          /* resident streams at most                              */
    int32_t max_sweeps_per_chunk; /* a chunk completes after this many sweeps at most      */
    int32_t sweeps_per_round;     /* batched sweeps per round                              */
    int32_t pad;
    double kkt_target;            /* relative KKT target of a chunk                        */
    double mixed_switch;          /* the mixed schedule's switch (as nmf_config)           */
    void *cuda_stream;            /* stream of the server's device work, or NULL           */
} nmf_server_config;

typedef struct {
    uint64_t ticket;              /* from nmf_server_submit                                */
    int32_t stream;
    int32_t ncols;                /* columns of the chunk                                  */
    double t_submit_s, t_done_s;  /* seconds since the server was created                  */
    int32_t sweeps;               /* sweeps the stream ran between the chunk's round and completion */
    int32_t converged;            /* 1: kkt_target met; 0: max_sweeps_per_chunk reached    */
    double kkt_rel, f;            /* of the stream's last measured iterate                 */
    int32_t m;                    /* resident columns of the stream at completion          */
    int32_t pad;
} nmf_chunk_result;

typedef struct {
    int64_t chunks_done, columns_done, rounds, batch_sweeps;
    int64_t stream_rounds;        /* sum over rounds of the streams swept in the round     */
    int32_t max_streams_in_round;
    int32_t streams_admitted, streams_queued, pad;
    int64_t hbm_in_use_bytes, hbm_budget_bytes;
} nmf_server_stats;

/* Defaults: hbm_budget 0 (90% of free memory), max_streams 64,
 * max_sweeps_per_chunk 500, sweeps_per_round 8, kkt_target 1e-6,
 * mixed_switch 1e-6. */
void nmf_server_config_init(nmf_server_config *cfg);

/* Start a server (and its worker thread) on the current device. */
nmf_status nmf_server_create(const nmf_server_config *cfg, nmf_server **out);

/* Stop the worker (chunks still in flight are dropped) and free everything. */
nmf_status nmf_server_destroy(nmf_server *s);

/* Open a stream of n rows, rank k (1..8 or 16) and m_capacity resident
 * columns; seed draws its U[0,1] starting factors.  The stream is queued for
 * admission (chunks may be submitted at once; they wait).  NMF_ECAPACITY if
 * its footprint alone exceeds the budget. */
nmf_status nmf_server_open_stream(nmf_server *s, int64_t n, int32_t k, int64_t m_capacity, uint64_t seed,
                                  int32_t *id);

/* Submit a chunk: ncols >= 1 FP32 host columns, column-major with leading
 * dimension ld >= n (copied before return).  *ticket (may be NULL)
 * identifies its result. */
nmf_status nmf_server_submit(nmf_server *s, int32_t id, const float *cols, int64_t ncols, int64_t ld,
                             uint64_t *ticket);

/* Close a stream once its chunks have completed (no more submissions). */
nmf_status nmf_server_close_stream(nmf_server *s, int32_t id);

/* Completed chunks, oldest first: up to cap results into out, their number
 * in *nout; waits up to wait_ms for the first one when none is ready. */
nmf_status nmf_server_poll(nmf_server *s, nmf_chunk_result *out, int32_t cap, int32_t *nout, int32_t wait_ms);

/* The stream's current factors (host buffers: X n x k, Y k x m with m the
 * resident columns, returned in *m; masks may be NULL), between rounds. */
nmf_status nmf_server_get_factors(nmf_server *s, int32_t id, double *X, double *Y, uint32_t *xmask,
                                  uint32_t *ymask, int64_t *m);

nmf_status nmf_server_get_stats(nmf_server *s, nmf_server_stats *out);
const char *nmf_server_last_error(nmf_server *s);

#ifdef __cplusplus
}
#endif

#endif /* NMF_GB300_H */
