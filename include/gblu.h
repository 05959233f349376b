/*
 * gblu -- sparse LU re-factorization with pivot check and sparse triangular
 * solves for circuit-simulation matrices, on one NVIDIA GB300 (sm_103a).
 *
 * The method is CKTSO's numerical path (arXiv 2411.14082):
 *   - factorization with pivoting (Section II-A, Algorithm 1), here in CSC
 *     form: left-looking column updates, threshold partial row pivoting;
 *   - fast re-factorization on the previous pattern and pivot order with a
 *     pivot check (Section IV-B, Algorithms 3 and 4), and, when a pivot fails
 *     the check, a restart that recomputes with pivoting the unfinished
 *     columns and their ancestors in the column elimination tree
 *     (Section IV-C and IV-D, Algorithm 5);
 *   - forward and back substitution (Section II-C, Algorithm 2, and the
 *     structure-adaptive parallel solve of Section V).
 * Ordering and symbolic analysis run on the host; all numerical work runs in
 * this library's CUDA kernels.  There is no CPU fallback.
 *
 * Conventions shared by every call
 *   - Matrices are CSC: Ap[n+1] (Ap[0] = 0, non-decreasing), Ai[nnz] row
 *     indices in [0, n), no duplicate row inside a column (rows inside a
 *     column may be unsorted), Ax[nnz] values (float64).  Indices are int32.
 *   - "_dev" pointers are device memory of the handle's device; other
 *     pointers are host memory.  The caller owns every pointer it passes;
 *     the library never frees caller memory and keeps no caller pointer after
 *     a call returns.  The handle owns its internal device buffers.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Kernels are queued on it; calls that must read a device result
 *     (documented below) synchronize that stream.
 *   - Return codes: GBLU_OK (0), GBLU_REPIVOTED (1, success after a restart
 *     with pivoting), or a negative GBLU_ERR_* code.  No call prints, aborts,
 *     or falls back to the CPU.  gblu_last_error() gives a one-line message.
 */
#ifndef GBLU_H
#define GBLU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBLU_OK 0
#define GBLU_REPIVOTED 1
#define GBLU_ERR_INVALID_INPUT (-1)  /* bad n, pointers, CSC pattern, duplicates, Q */
#define GBLU_ERR_SINGULAR (-2)       /* a column has no nonzero pivot candidate     */
#define GBLU_ERR_NOT_ANALYZED (-3)   /* call order violated                         */
#define GBLU_ERR_NOMEM (-4)          /* device or host allocation failed            */
#define GBLU_ERR_DEVICE_TIMEOUT (-5) /* a bounded device wait ran out               */
#define GBLU_ERR_CUDA (-6)           /* a CUDA runtime call failed                  */
#define GBLU_ERR_NOT_FACTORIZED (-7) /* refactorize/solve before a factorization    */
#define GBLU_ERR_INTERNAL (-8)       /* a structural invariant check failed         */
#define GBLU_ERR_BUSY (-9)           /* a server request has not finished yet       */
#define GBLU_ERR_NONFINITE (-10)     /* a NaN or infinite value reached a pivot column */

/* Scheduling of the re-factorization (Section IV-B: cluster and pipeline modes). */
#define GBLU_SCHED_AUTO 0     /* level-synchronous front, sync-free tail      */
#define GBLU_SCHED_LEVEL 1    /* every level a separate launch (cluster mode) */
#define GBLU_SCHED_SYNCFREE 2 /* one launch, ready flags (pipeline mode)      */

typedef struct gblu_ctx *gblu_handle;

typedef struct {
    double pivot_tol;    /* eps of the pivot rule |x(k)| >= eps*max|x(L rows)|
                            (Section II-A; the paper gives no value), default 1e-3 */
    int sched_mode;      /* GBLU_SCHED_*, default AUTO                            */
    int solve_mode;      /* GBLU_SCHED_*, same meaning for the triangular solves  */
    double alpha;        /* dividing level = first level with fewer than
                            alpha * resident warps columns (Section IV-B uses
                            alpha = 2 per thread), default 2.0                    */
    long long spin_limit;/* iterations of every device wait before it gives up
                            with GBLU_ERR_DEVICE_TIMEOUT, default 1<<24           */
    /* structure-adaptive solve (Section V-A): the trailing block L(P0:n,P0:n)
       (and U likewise) is split off when it holds at least solve_dense_frac
       of the factor's entries and at least solve_dense_min entries (the
       paper's rule: 0.7, 300000).  solve_dense_density > 0 retunes the rule
       for the GPU: P0 is then the start of the longest trailing block whose
       entry density stays at least that value (solve_dense_frac ignored);
       default 0.9.  The block is solved in trapezoid slices of 32 rows, one
       warp each, sync-free (Section V-B); solve_slices is the number of
       slices of equal entry counts reported by gblu_get_stats for the
       paper's own cut, and solve_slices = 0 disables the split.           */
    double solve_dense_frac;
    long long solve_dense_min;
    int solve_slices;
    double solve_dense_density;
    /* dense tail of the re-factorization: when the last m columns of the
       factor form a structurally dense block (every column k >= n-m holds
       every row >= n-m) and m >= dense_min_rows, the re-factorization applies
       the sparse dependencies of those columns in the column kernels and
       then factors the block as a dense matrix (blocked right-looking, the
       same pivot check per column, no row interchanges); at most
       GBLU_DENSE_MAX_ROWS rows are taken.  0 disables it (the default: on
       the 200x200x4 mesh its one-SM panels cost more than the column
       kernels do on the same block).                                        */
    int dense_min_rows;
    /* warp assignment of the re-factorization (Section IV-B's task
       granularity, retuned for warps): columns of at most warp_column_max
       entries are computed by one warp (eight per CTA), longer ones by half
       a CTA (up to 2560 entries) or a whole CTA.  32..640, default 640;
       gblu_autotune measures it. */
    int warp_column_max;
    /* first factorization (gblu_factorize, Algorithm 1 with the threshold
       rule and the diagonal row A(Q[k],Q[k]) preferred):
       2 = the prediction that every step keeps its diagonal row becomes a
       structure (gblu_symmetric_structure) that is installed, and the
       checked re-factorization kernel computes every column on it; when a
       check fails, the threshold rule's row at the first failing step is
       exchanged with the row of the step that held it and the structure is
       predicted again (as a restart on a predicted structure does, see
       gblu_refactorize); after six such rounds, a round without progress or
       a non-finite candidate, every step goes through the pivoting kernel
       as in 1.  Taken when every column of A has a
       nonzero diagonal entry and at most 2% of the off-diagonal entries of
       A lack their transposed entry; otherwise as 1.
       1 = the pivoting kernel's passes speculate that each step pivots on
       its diagonal row and wait only on the steps that prediction names as
       dependencies; steps after the first one that took another row run
       again, and the run falls back to waiting on every earlier unfinished
       step of the column's elimination subtree once more than four finished
       steps of a pass have left the diagonal, a pass finishes no step for
       good, or eight passes have run.  It does not speculate at all when
       more than four columns of A have an absent or zero diagonal entry.
       0 = every step waits in that order from the start.  All three give
       the same pivots and factor values (2 may store exact zeros at the
       extra positions of its structure).  Default 2. */
    int speculate_first;
    /* batches of value sets (gblu_refactorize_batch): the persistent launch
       takes the sets in groups of batch_group, all tasks of one group before
       the next group's, so that the factors being read stay in L2 (0 = as
       many sets as fit in half of L2; >= nsets: every set at once).
       Default 0. */
    int batch_group;
    /* CTAs (8 warps each) per SM of the sync-free solve launches; 0 = as
       many as fit.  Fewer resident warps poll fewer unpublished values at a
       time.  gblu_autotune measures it. */
    int solve_ctas_per_sm;
    /* SMs the handle's persistent launches (re-factorization, pivoting,
       sync-free solves) may use; 0 = all.  A server gives its large patterns
       part of the device so that small requests run beside them. */
    int max_sms;
} gblu_opts;

/* largest dense tail block of the re-factorization (shared-memory panel) */
#define GBLU_DENSE_MAX_ROWS 3456

/* Fill *o with the defaults above. */
void gblu_default_opts(gblu_opts *o);

/*
 * gblu_get_opts: the handle's current options.
 * gblu_set_opts: replace them; on a factorized handle the schedule of the
 *   re-factorization and the solves is rebuilt for the same factor
 *   structure and values (host work, then an upload on `stream`, which is
 *   synchronized).  GBLU_ERR_INVALID_INPUT for out-of-range options.
 * gblu_autotune: measure, with CUDA events on `stream`, the median of reps
 *   re-factorizations of Ax_dev and solves of b_dev (into x_dev) for a set
 *   of schedule options, and keep the fastest: first the dividing-level
 *   factor alpha (Section IV-B) and the warp assignment (warp_column_max)
 *   by re-factorization time, then the trailing-block rule of the solve
 *   (solve_dense_density, and solve_slices = 0 to disable it; Section
 *   V-A) and the resident CTAs of the sync-free solves
 *   (solve_ctas_per_sm) by solve time.  The paper tunes these constants for its
 *   CPUs; here they are measured on the device and matrix at hand.  The
 *   factor values after the call are those of Ax_dev.  *chosen, *refactor_ms
 *   and *solve_ms (optional, host) report the kept options and their times.
 */
int gblu_get_opts(gblu_handle h, gblu_opts *o);
int gblu_set_opts(gblu_handle h, const gblu_opts *o, void *stream);
int gblu_autotune(gblu_handle h, const double *Ax_dev, const double *b_dev, double *x_dev, int32_t reps,
                  void *stream, gblu_opts *chosen, double *refactor_ms, double *solve_ms);

/* One-line description of the last error of this thread (never NULL). */
const char *gblu_last_error(void);

/* Create a handle on CUDA device `device`; o may be NULL for defaults.
 * Returns GBLU_ERR_CUDA if the device cannot be used. */
int gblu_create(gblu_handle *h, int device, const gblu_opts *o);

/* Release every device buffer of the handle (synchronizes the device). */
void gblu_destroy(gblu_handle h);

/*
 * Pre-processing for one sparsity pattern (Section III-A): validates the CSC
 * pattern, takes the column order Q (Q[k] = original column eliminated at
 * step k; rows use the same symmetric order as the preferred pivots), or
 * when Q is NULL computes its own fill-reducing order on A+A^T
 * (gblu_order_auto), and builds the column elimination tree of A(:,Q) (the dependency upper bound of
 * Section II-B used to choose restart columns).  Host-only work.  Ap, Ai,
 * Q are host arrays and are copied.  Any previous factorization of the
 * handle is discarded.
 */
int gblu_analyze(gblu_handle h, int32_t n, const int32_t *Ap, const int32_t *Ai,
                 const int32_t *Q);

/*
 * Factorization with pivoting (Section II-A, Algorithm 1 in CSC form, run as
 * the pipelined factorization of Section IV-D over all columns: columns are
 * taken in increasing order, and each waits only for earlier columns of its
 * column-elimination subtree).  Every step prefers its diagonal row Q[k] and
 * keeps it unless |x(Q[k])| < pivot_tol * max|other candidates| or
 * x(Q[k]) == 0, else takes the largest candidate (ties: the row first in Q).
 * By default (speculate_first = 2) the prediction that every step keeps its
 * diagonal row is first installed as a structure and the checked
 * re-factorization kernel computes the columns on it; where a check fails,
 * the pivot moves by re-prediction (see gblu_refactorize), or, when that
 * gives up, the pivoting kernel computes every step.
 * Ax_dev: device float64[nnz] in the slot order of the analyze call's Ai.
 * Builds the factors and, on the host, the fixed-pattern schedule for
 * refactorize and solve.  Synchronizes `stream`.
 * Returns GBLU_OK, GBLU_ERR_SINGULAR or GBLU_ERR_NONFINITE (a NaN or
 * infinite value in a column; factors then invalid).
 */
int gblu_factorize(gblu_handle h, const double *Ax_dev, void *stream);

/*
 * Fast re-factorization with pivot check (Section IV, Algorithms 3-5):
 * recomputes the factors of new values on the previous pattern and pivot
 * order, checking every pivot.  If a pivot fails, the restart recomputes
 * with pivoting, preferring the previous pivots.  On a structure the
 * pivoting kernel produced (and after a forced failure, see
 * gblu_refactorize_forced) it first runs the unfinished columns again on
 * the installed structure, speculating that every step keeps its preferred
 * row, with the same check confirming each (exact when all pass: the
 * structure is then the old one); if a check fails again, a pivot must
 * move.  On a structure that was predicted (the first factorization's, or
 * a re-prediction's), that first stage could only fail again, so the
 * re-factorization itself runs without stopping at a failed check (later
 * columns are recomputed anyway) and a failure goes straight to the pivot
 * move: the first failing step takes the
 * threshold rule's row, the step that held that row takes the failing
 * step's row, the structure is predicted again for these pivot rows (the
 * Cholesky pattern of B + B^T with B = A(piv, Q), which holds the factors
 * of B without exchanges) and every column is re-factorized on it with the
 * check; a step whose preferred row went elsewhere must then pivot on its
 * largest candidate.  Up to six rounds, each moving the first failure
 * forward; if they do not finish, every step goes through the pivoting
 * kernel.  On another structure, the unfinished columns and their
 * elimination-tree ancestors go through the pivoting kernel.  Either way
 * the schedule is rebuilt.  The call then
 * returns GBLU_REPIVOTED.  The result equals a factorization with pivoting that
 * prefers the previous pivot sequence.  Synchronizes `stream` once (to read
 * the 4-byte check status).  *repivoted (optional, host) is set to 1 if a
 * restart happened, else 0.  A NaN or infinite pivot or entry of L fails
 * the check; the restart then returns GBLU_ERR_NONFINITE instead of storing
 * it in the factors (a NaN that stays in U shows in gblu_residual).
 */
int gblu_refactorize(gblu_handle h, const double *Ax_dev, void *stream,
                     int32_t *repivoted);

/*
 * gblu_refactorize with the pivot check of step force_col treated as failed
 * whatever its value (force_col = -1: none), so that the restart runs from
 * that step: the protocol of the paper's general-case evaluation (Section
 * VI-A), where selected runs re-pivot at a random row.  With unchanged
 * values the restart keeps the previous pivots.  A step inside the dense
 * tail block (dense_min_rows > 0) is not forced.  Returns as
 * gblu_refactorize; GBLU_ERR_INVALID_INPUT if force_col is outside [-1, n).
 */
int gblu_refactorize_forced(gblu_handle h, const double *Ax_dev, void *stream, int32_t force_col,
                            int32_t *repivoted);

/*
 * One Newton step on device buffers, replayed from a CUDA graph: the
 * checked re-factorization of Ax_dev (as gblu_refactorize) and the solve of
 * b_dev into x_dev, with one synchronization at the end instead of one
 * between the two.  The graph (staging copies of Ax and b, all launches of
 * the refactorization, the status copy and the solve) is captured on the
 * first call and again after the structure changes.  The solve runs before
 * the check status is known; if a check failed, the call restarts with
 * pivoting and solves again (returns GBLU_REPIVOTED, *repivoted = 1).
 * Results equal gblu_refactorize + gblu_solve.  x_dev must not alias b_dev.
 */
int gblu_step(gblu_handle h, const double *Ax_dev, const double *b_dev, double *x_dev, void *stream,
              int32_t *repivoted);

/*
 * Solve A x = b with the current factors: y = L^-1 P b, z = U^-1 y,
 * x(Q) = z (Algorithm 2 and the parallel solve of Section V).  b_dev and
 * x_dev are device float64[n]; they may alias.  Asynchronous on `stream`.
 */
int gblu_solve(gblu_handle h, const double *b_dev, double *x_dev, void *stream);

/*
 * Status of the handle's last device work, after synchronizing `stream`
 * (the device status word of Section IV's pivot check and waits, latched
 * in the handle's control block until the next call resets it): the error
 * the device recorded (GBLU_ERR_DEVICE_TIMEOUT, GBLU_ERR_SINGULAR, ...), or
 * else GBLU_REPIVOTED when the last gblu_refactorize / gblu_step restarted
 * with pivoting, else GBLU_OK.  The numeric calls already return these
 * codes; this reads them again without new work.
 */
int gblu_last_status(gblu_handle h, void *stream);

/*
 * Batch of value sets on the installed structure (many same-pattern systems,
 * e.g. the Newton iterations of independent simulations of one circuit): the
 * checked re-factorization of Algorithms 3 and 4 for every set, in one
 * persistent launch that reads the structure once.  The paper works on one
 * matrix at a time; batching is this library's extension.
 *   Ax_dev   device float64, set s at Ax_dev + s*ax_stride, each in the CSC
 *            slot order of gblu_analyze (ax_stride >= nnz(A));
 *   LUx_dev  device float64, set s at LUx_dev + s*lu_stride (lu_stride >=
 *            nnz_l + nnz_u of gblu_get_stats): receives the set's factor
 *            values in the handle's internal layout; read them back only
 *            through gblu_solve_batch.  Caller-owned.
 *   failed   optional host int32[nsets]: 1 if a pivot of that set failed
 *            the check, else 0.  A failed set is not restarted (a restart
 *            changes the set's pattern): its values are not valid, and it
 *            must be factorized on a handle of its own.  Other sets are not
 *            affected.
 *   n_failed optional host: number of failed sets.
 * The handle's own factors are not touched.  Synchronizes `stream` once.
 * Errors: GBLU_ERR_INVALID_INPUT (nsets < 1, null buffer, small stride),
 * GBLU_ERR_NOT_FACTORIZED, GBLU_ERR_DEVICE_TIMEOUT.
 */
int gblu_refactorize_batch(gblu_handle h, int32_t nsets, const double *Ax_dev, int64_t ax_stride,
                           double *LUx_dev, int64_t lu_stride, int32_t *failed, int32_t *n_failed,
                           void *stream);

/*
 * Solve A_s x_s = b_s for every set of a batch whose factor values came from
 * gblu_refactorize_batch (sets that failed give meaningless x).  b and x are
 * device float64, set s at b_dev + s*b_stride, x_dev + s*x_stride (strides
 * >= n; b and x may alias).  Asynchronous on `stream`.
 */
int gblu_solve_batch(gblu_handle h, int32_t nsets, const double *LUx_dev, int64_t lu_stride,
                     const double *b_dev, int64_t b_stride, double *x_dev, int64_t x_stride,
                     void *stream);

/*
 * gblu_refactorize_batch followed by gblu_solve_batch, replayed from one
 * CUDA graph (this library's extension of the batched form; the paper runs
 * one matrix at a time).  Arguments and results as in those two calls: the
 * sets' values at Ax_dev + s*ax_stride, factor values written at LUx_dev +
 * s*lu_stride, right-hand sides at b_dev + s*b_stride, solutions at x_dev +
 * s*x_stride; failed[s] / *n_failed (optional host) as in
 * gblu_refactorize_batch, and the x of a failed set is not valid.
 * The first call with a given set count, buffer addresses and strides (or
 * after the structure or the handle's device buffers changed) runs the two
 * calls eagerly and captures them; later calls with the same arguments
 * replay the graph: one launch of every kernel, one synchronization of
 * `stream`, and a read of the sets' control blocks.  The buffers' contents
 * may change between calls; their addresses must not.  Errors as in
 * gblu_refactorize_batch, plus GBLU_ERR_CUDA if the capture fails.
 */
int gblu_step_batch(gblu_handle h, int32_t nsets, const double *Ax_dev, int64_t ax_stride,
                    double *LUx_dev, int64_t lu_stride, const double *b_dev, int64_t b_stride,
                    double *x_dev, int64_t x_stride, int32_t *failed, int32_t *n_failed,
                    void *stream);

/*
 * Batch over handles of DIFFERENT patterns (this library's extension): the
 * checked re-factorization of Algorithms 3 and 4 for every handle hs[i]
 * with its own values Ax_dev[i] (device, its analyze slot order), into that
 * handle's own factors, in one persistent launch.  The handles' tasks share
 * one ticket queue: each handle's tasks keep their topological order and
 * the handles are interleaved so that they advance at the same relative
 * pace.  A handle whose check fails then restarts alone, as in
 * gblu_refactorize (Section IV-C); repivoted (optional, host int32[nh]) is
 * 1 for those.  All handles must be factorized, distinct and on one device.
 * The launch runs on `stream` and the call synchronizes it once (plus once
 * per restart).  Results equal those of gblu_refactorize on each handle.
 * gblu_solve_multi: gblu_solve for every handle, b_dev[i] -> x_dev[i],
 * asynchronous on `stream`.
 */
int gblu_refactorize_multi(int32_t nh, gblu_handle *hs, const double *const *Ax_dev, void *stream,
                           int32_t *repivoted);
int gblu_solve_multi(int32_t nh, gblu_handle *hs, const double *const *b_dev, double *const *x_dev,
                     void *stream);

/*
 * Mixed precision (this library's extension; the paper factors in double).
 *
 * gblu_refactorize_f32: the checked re-factorization of Algorithms 3 and 4
 * computed in single precision (A values are rounded once when scattered;
 * the pivot check compares single-precision values) into a separate factor
 * array of the handle.  The handle's double-precision factors are not
 * touched.  *check_failed (optional, host) = 1 if a pivot failed the check:
 * those factors are then not used, and gblu_solve_refined falls back to
 * double precision.  Synchronizes `stream` once.
 *
 * gblu_solve_refined: solves A x = b for the A values Ax_dev (the CSC slot
 * order of gblu_analyze) by iterative refinement on the single-precision
 * factors of the last gblu_refactorize_f32: x = solve(b), then while the
 * backward error ||b - A x||inf / (||A||inf ||x||inf), computed in double, is
 * above tol: x += solve(b - A x).  The solves run in double on the widened
 * factors.  If the error does not halve in an iteration, max_iter corrections
 * are used up, or the factors failed the check, it re-factorizes in double
 * precision (gblu_refactorize, with its restart) and solves directly:
 * *iters (optional, host) is then -1, else the number of corrections.
 * *berr (optional, host) = the final backward error.  x_dev must not alias
 * b_dev.  Synchronizes `stream` once per iteration.
 */
int gblu_refactorize_f32(gblu_handle h, const double *Ax_dev, void *stream, int32_t *check_failed);
int gblu_solve_refined(gblu_handle h, const double *Ax_dev, const double *b_dev, double *x_dev, double tol,
                       int32_t max_iter, void *stream, int32_t *iters, double *berr);

/*
 * Relative residual of a solution, computed on the device in float64:
 * out_dev[0] = ||b - A x||_inf / (||A||_inf * ||x||_inf), out_dev[1] =
 * ||b - A x||_inf, out_dev[2] = ||A||_inf, out_dev[3] = ||x||_inf.
 * Ax_dev uses the analyze slot order.  Asynchronous on `stream`.
 * (A measurement aid; not part of the paper's method.)
 */
int gblu_residual(gblu_handle h, const double *Ax_dev, const double *b_dev,
                  const double *x_dev, double *out_dev, void *stream);

/*
 * One Newton-Raphson linear step from HOST buffers: copies Ax_host (nnz
 * values, analyze slot order) and b_host (n) to handle-owned device staging
 * buffers, re-factorizes with pivot check (as gblu_refactorize), solves, and
 * copies the solution to x_host (n).  Host buffers may be pageable; pinned
 * buffers make the copies asynchronous.  Synchronizes `stream` before
 * returning.  Returns what gblu_refactorize returns (GBLU_OK or
 * GBLU_REPIVOTED) or an error.
 */
int gblu_step_host(gblu_handle h, const double *Ax_host, const double *b_host,
                   double *x_host, void *stream, int32_t *repivoted);

/*
 * Allocation-free solve for callers that cannot allocate device memory (a
 * simulator that runs on its own fixed device pool, code running while a
 * CUDA graph is being captured, builds that forbid allocation after
 * start-up).  The paper has no counterpart; this is an interface
 * convenience.  It solves A x = b from factors the caller keeps in its own
 * device buffers, with sync-free row solves like gblu_solve's, and
 * allocates nothing: its scratch (intermediate vector, ready flags,
 * tickets) is one file-scope device array of 8 MB, held on a device from
 * the time the library's module is loaded there until the process exits.
 *   Factors, row-wise (CSR) in step numbering, all device arrays:
 *   Lrp[n+1]/Lcol/Lval = strict lower part of L (unit diagonal implied),
 *   Urp[n+1]/Ucol/Uval = strict upper part of U, Udiag[n] = U(k,k),
 *   piv[n] = original row of step k, q[n] = original column of step k
 *   (gblu_export_factors gives the same factors column-wise).
 *   b_dev[n] -> x_dev[n] (must not alias); status_dev (optional device
 *   int32) receives 0 or GBLU_ERR_DEVICE_TIMEOUT when the solve finishes.
 *   The return code only covers the launches: without status_dev a wait
 *   that ran out (x_dev then partly written) cannot be seen.
 *   spin_limit: polls of one ready flag before the wait gives up (<= 0:
 *   2^24).
 * n must be <= GBLU_NOALLOC_MAX_N; larger n returns GBLU_ERR_INVALID_INPUT
 * with a message.  Asynchronous on `stream`.  Within one process every call
 * on a device shares the scratch array (it keeps the last call's contents;
 * each call clears its flags first): calls that overlap on the GPU
 * (different streams or host threads) race, so serialize them.  Each call
 * looks up the array's device address with the current device; the first
 * call on a device also queries the occupancy, so make it before any stream
 * capture.
 */
#define GBLU_NOALLOC_MAX_N 524288
int gblu_solve_factors_noalloc(int32_t n, const int64_t *Lrp, const int32_t *Lcol,
                               const double *Lval, const int64_t *Urp, const int32_t *Ucol,
                               const double *Uval, const double *Udiag, const int32_t *piv,
                               const int32_t *q, const double *b_dev, double *x_dev,
                               int32_t *status_dev, long long spin_limit, void *stream);

/*
 * Solve server (this library's extension; the paper solves one matrix at a
 * time).  A server on one device keeps one handle resident per registered
 * pattern and answers requests "solve A x = b for these values of pattern
 * p".  Per pattern a worker thread with its own stream takes the queued
 * requests, up to the pattern's slot count, and runs them as one batch
 * (gblu_refactorize_batch + gblu_solve_batch); requests that arrive while a
 * batch runs go into the next one.  Patterns overlap on the device.  A
 * request whose pivot check fails is redone with gblu_refactorize (restart
 * with pivoting, Section IV-C), and the pattern keeps the new pivot
 * sequence.  Each result is bit-for-bit the result of the same request run
 * alone on a handle in the same pivot state.  A pattern of more than
 * 100,000 unknowns gets max_sms = 3/4 of the SMs and a low-priority stream;
 * the others get high-priority streams, so that small requests start beside
 * a large one's persistent launches.  Request values, right-hand sides and
 * solutions pass through pinned host buffers of the server (a copy to or
 * from pageable memory would queue behind other streams' copies in the
 * driver's shared staging).  Streams share the device's hardware
 * work queues (8 by default): a process serving many patterns should set
 * CUDA_DEVICE_MAX_CONNECTIONS=32 before it creates its CUDA context, or a
 * short launch can wait in a queue behind a long one of another pattern.
 *
 * gblu_server_create: budget = device bytes the server may hold in total;
 *   max_batch = most requests per batch; o = options of the handles (NULL:
 *   defaults).
 * gblu_server_add_pattern: analyze (Q may be NULL, as in gblu_analyze) and
 *   factorize with pivoting on the first values Ax0_host (host, nnz(A), slot
 *   order of Ai); then admits the pattern only if its footprint (handle:
 *   structure, factors, workspace; plus batch buffers) fits in what is left
 *   of the budget.  *slots = the largest batch that fits (<= max_batch).
 *   Returns GBLU_ERR_NOMEM when even one slot does not fit, or the error of
 *   the analysis or factorization.  Synchronizes the device.
 * gblu_server_submit: queues a request.  Ax_host (nnz(A), slot order),
 *   b_host (n) and x_host (n) are host arrays owned by the caller and must
 *   stay valid until the request is waited for; x_host receives the
 *   solution.  Pinned host memory makes the copies asynchronous.  mode 0:
 *   double precision (batched); mode 1: single-precision factors with
 *   refinement to a backward error of 1e-12 (gblu_refactorize_f32 +
 *   gblu_solve_refined, one request at a time, falling back to double
 *   precision when refinement stalls).
 * gblu_server_wait: waits up to timeout_s seconds (0: poll).  Returns
 *   GBLU_OK and fills *res (then the request id is released), or
 *   GBLU_ERR_BUSY if it has not finished.  res->status is the request's own
 *   outcome: GBLU_OK, GBLU_REPIVOTED or an error code.
 * gblu_server_pattern_info: a pattern's slots, device footprint and factor
 *   entries (nnz(L) + nnz(U)); each output optional.
 * gblu_server_destroy: finishes every queued request, stops the workers and
 *   frees all device memory of the server.
 * Errors of these calls are described by gblu_server_last_error().
 */
typedef struct gblu_server_s *gblu_server;

typedef struct {
    int32_t status;      /* GBLU_OK, GBLU_REPIVOTED or an error code              */
    int32_t repivoted;   /* 1 if its check failed and it was redone with pivoting */
    int32_t batch_size;  /* requests in the batch it ran in                       */
    int32_t pattern;
    double berr;         /* ||b - A x||inf / (||A||inf ||x||inf); -1 on error     */
    double queue_s;      /* submit -> start of its batch (host clock)             */
    double latency_s;    /* submit -> solution in x_host (host clock)             */
    int32_t refine_iters;/* mode 1: corrections used, -1 = fell back to double    */
} gblu_request_result;

typedef struct {
    int64_t budget_bytes, reserved_bytes;
    int32_t n_patterns;
    int32_t max_batch_seen;
    int64_t submitted, completed, batches, repivots;
} gblu_server_stats;

const char *gblu_server_last_error(void);
int gblu_server_create(gblu_server *s, int device, int64_t hbm_budget_bytes, int32_t max_batch,
                       const gblu_opts *o);
int gblu_server_add_pattern(gblu_server s, int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *Q,
                            const double *Ax0_host, int32_t *pattern, int32_t *slots);
int gblu_server_pattern_info(gblu_server s, int32_t pattern, int32_t *slots, int64_t *footprint_bytes,
                             int64_t *nnz_lu);
int gblu_server_submit(gblu_server s, int32_t pattern, const double *Ax_host, const double *b_host,
                       double *x_host, int32_t mode, int64_t *request);
int gblu_server_wait(gblu_server s, int64_t request, double timeout_s, gblu_request_result *res);
int gblu_server_get_stats(gblu_server s, gblu_server_stats *st);
void gblu_server_destroy(gblu_server s);

/*
 * Static pivoting and scaling (the optional pre-processing of Section
 * III-A).  Host-only.
 * gblu_static_pivot: a row permutation maximizing the product of the
 *   diagonal magnitudes, with scalings that make the matched entries 1 and
 *   every entry at most 1 in magnitude.  match[j] = the row of A placed on
 *   the diagonal in column j (so (P A)(j, :) = A(match[j], :));
 *   row_scale[i], col_scale[j] (optional) = Dr, Dc with
 *   |Dr[i] a_ij Dc[j]| <= 1 and = 1 where i = match[j].  Entries stored
 *   with value 0 are not used.  GBLU_ERR_SINGULAR if no perfect matching
 *   exists on the nonzero entries.
 * gblu_permute_rows: the CSC pattern of P A: Ai_out[e'] (rows sorted in
 *   each column) and src_out[e'] = the entry of A that lands in slot e'.
 * The scaled system Dr P A Dc y = Dr P b gives x = Dc y.  Per value set,
 * Ax'[e'] = Ax[src[e']] * Dr[Ai[src[e']]] * Dc[j] and b'[j] =
 * b[match[j]] * Dr[match[j]] are one gblu_gather_scale each, and so is
 * x = Dc * y (src = NULL).
 * gblu_gather_scale: out[k] = in[src[k]] * scale[k] for k < m, on the
 *   device (src NULL: in[k]; scale NULL: 1).  Asynchronous on `stream`.
 */
int gblu_static_pivot(int32_t n, const int32_t *Ap, const int32_t *Ai, const double *Ax, int32_t *match,
                      double *row_scale, double *col_scale);
int gblu_permute_rows(int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *match, int32_t *Ai_out,
                      int32_t *src_out);
int gblu_gather_scale(int64_t m, const int32_t *src_dev, const double *scale_dev, const double *in_dev,
                      double *out_dev, void *stream);

/* Sizes and counters of the current factorization (host struct). */
typedef struct {
    int32_t n;
    int64_t nnz_a;
    int64_t nnz_l;        /* strict lower entries                            */
    int64_t nnz_u;        /* upper entries incl. diagonal                    */
    double flops;         /* refactor flops: sum over updates 2*nnz(L(:,j))   */
    int32_t n_levels;     /* levels of the column dependency graph (EGraph)  */
    int32_t div_level;    /* first level scheduled sync-free                 */
    int32_t n_solve_levels_l, n_solve_levels_u;  /* levels of the sparse blocks     */
    int32_t solve_p0_l, solve_p0_u;  /* first row of the trailing dense block (n: none) */
    int32_t solve_slices_l, solve_slices_u;  /* the paper's slices of the trailing block */
    int32_t etree_height;
    int64_t n_refactor;   /* refactorize calls                               */
    int64_t n_repivot;    /* refactorize calls that restarted with pivoting  */
    int64_t n_restart_cols; /* columns recomputed by the last restart        */
    int32_t last_first_bad; /* first failing column of the last check, -1    */
    int64_t device_bytes; /* device memory held by the handle                */
    int64_t kernel_launches; /* kernels this handle has launched so far      */
    int32_t dense_rows;   /* rows of the dense tail block (0: none)          */
    /* last factorization with pivoting (first factorization or restart),
     * host wall clock: tail kernel, download and repack of the factors,
     * schedule rebuild, upload of the new structure.  On a predicted
     * structure the solve part of the schedule is built on the host while
     * the re-factorization runs; it counts in tail_schedule_ms and in
     * tail_kernel_ms (the re-factorization's wall clock), and its upload
     * in tail_kernel_ms only. */
    double tail_kernel_ms, tail_repack_ms, tail_schedule_ms, tail_upload_ms;
    int32_t tail_passes;  /* kernel passes of that run (a restart speculates
                             that the preferred pivots are kept and repeats
                             the steps after a step that took another row);
                             0: the restart's first stage, the unfinished
                             columns re-factorized on the installed
                             structure with the check, kept every pivot
                             (tail_kernel_ms is then that stage's time) */
    /* last gblu_factorize: 0 = the pivoting kernel computed every step;
       1 = the checked re-factorization on the predicted structure passed
       every check (tail_kernel_ms is its time, first_symbolic_ms the
       structure's on the host); 3 = a check failed there and re-predicted
       structures (repredictions of them) completed the factorization;
       2 = the re-prediction gave up and the pivoting kernel computed every
       step (the tail_* fields describe it) */
    int32_t first_mode;
    double first_symbolic_ms;
    /* wide columns of the installed structure (at most 64 L entries, at
       least 256 supernode runs among the dependencies): the re-factorization
       applies all but their last run of dependencies row by row through the
       rows of L (0 when the per-CTA scratch would exceed 1 GiB) */
    int64_t wide_cols;
    /* structure re-predictions of the last restart or first factorization
       on a predicted structure: each is one pivot exchange found by the
       threshold rule at the first failing step, a new predicted structure
       (the Cholesky pattern of B + B^T for B = A with the new pivot rows)
       and one checked re-factorization of every column (0: none needed) */
    int32_t repredictions;
} gblu_stats;

int gblu_get_stats(gblu_handle h, gblu_stats *s);

/*
 * Measurement aid (not part of the paper's method): the FP64 fused
 * multiply-add rate of `device`, the roof of the re-factorization, which
 * runs on the non-tensor FP64 pipe.  Times a kernel of eight independent
 * multiply-add chains per thread on every SM (best of three after a warm-up
 * run) and writes TFLOP/s (2 flops per multiply-add) to *tflops (host).
 * Allocates and frees a small device buffer; synchronizes the device.
 * Returns GBLU_OK, GBLU_ERR_INVALID_INPUT (tflops NULL) or GBLU_ERR_CUDA.
 */
int gblu_fp64_fma_rate(int device, double *tflops);

/*
 * Copy the current factors to host arrays (for verification): column k of
 * L (strict lower) and U (upper, diagonal last) in step numbering with rows
 * sorted, piv[k] = original row pivotal at step k, q[k] = original column
 * of step k.  Array sizes: Lp/Up n+1, Li/Lx nnz_l, Ui/Ux nnz_u, piv/q n.
 * Any pointer may be NULL to skip it.  Synchronizes the device.
 */
int gblu_export_factors(gblu_handle h, int64_t *Lp, int32_t *Li, double *Lx,
                        int64_t *Up, int32_t *Ui, double *Ux, int32_t *piv,
                        int32_t *q);

/*
 * Host-only helpers (no device work), exposed so that the symbolic layer can
 * be checked on machines without a GPU.  Common to all of them: Ap, Ai (a
 * CSC pattern, columns in any row order) and every other argument are host
 * arrays owned by the caller, read or written only during the call; perm
 * and other outputs have n entries.  An invalid pattern (n < 1, Ap[0] != 0,
 * Ap decreasing, a row index outside [0, n), a duplicate entry in a column)
 * or a null output gives GBLU_ERR_INVALID_INPUT and writes nothing.
 */
/* Minimum-degree column order of the pattern of A + A^T: perm[k] = column
 * eliminated at step k. */
int gblu_order_mindeg(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm);
/* Approximate minimum deficiency on the pattern of A + A^T (the minimum
 * degree variant Section III-A also runs): each step eliminates the vertex
 * whose elimination is estimated to add the fewest entries,
 * d(d-1)/2 - c(c-1)/2 with d its approximate degree and c+1 the size of the
 * largest clique (element) it belongs to; ties to the lower index. */
int gblu_order_amf(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm);
/* Constrained minimum degree (the ordering Section III-A applies after an
 * incomplete nested dissection): group[i] >= 0 for every vertex; the
 * vertices are eliminated group by group in increasing group number, and
 * within a group by least approximate degree in the whole graph (ties to
 * the lower index).  With one group it equals gblu_order_mindeg. */
int gblu_order_cmd(int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *group, int32_t *perm);
/* Nested dissection column order of the pattern of A + A^T, without
 * coordinates (multilevel: heavy-edge coarsening, greedy growing bisection,
 * boundary refinement, vertex cover of the cut edges as separator; sets of
 * at most 256 vertices by minimum degree).  Deterministic. */
int gblu_order_nd(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm);
/* Incomplete nested dissection followed by constrained minimum degree
 * (Section III-A): the dissection of gblu_order_nd only assigns groups (each
 * set of at most 256 vertices, then each separator after its two halves),
 * and one minimum-degree pass orders the whole graph, taking the groups in
 * that order, so leaf orders see their boundaries and separators are
 * ordered as well.  Deterministic. */
int gblu_order_cnd(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm);
/* methods of gblu_order_auto */
#define GBLU_ORDER_MINDEG 0   /* gblu_order_mindeg */
#define GBLU_ORDER_ND 1       /* gblu_order_nd     */
#define GBLU_ORDER_CND 2      /* gblu_order_cnd    */
#define GBLU_ORDER_AMF 3      /* gblu_order_amf    */
/* Section III-A's selection: several orders are computed on host threads
 * (minimum degree, approximate minimum deficiency and nested dissection
 * with constrained minimum degree up to n = 200000, nested dissection at
 * every size), and the one whose factorization costs
 * the fewest flops when every diagonal pivot is kept (gblu_symmetric_cost)
 * is written to perm; ties go to that list's order.  *method (optional)
 * receives its GBLU_ORDER_* code.  gblu_analyze uses it when Q is NULL. */
int gblu_order_auto(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm, int32_t *method);
/* Entries of the strict lower Cholesky factor of (A + A^T)(Q,Q): the fill of
 * an ordering when every diagonal pivot is kept; negative on invalid input. */
int64_t gblu_symmetric_fill(int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *Q);
/* The same fill (*fill, optional) and the factorization's flops when every
 * diagonal pivot is kept on that symmetric pattern, F = sum_j 2 c_j^2 with
 * c_j the entries of column j (*flops, optional).  GBLU_ERR_INVALID_INPUT
 * for an invalid pattern or a Q that is not a permutation. */
int gblu_symmetric_cost(int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *Q, int64_t *fill,
                        double *flops);
/* The factor structure that gblu_factorize predicts before its first
 * factorization (Algorithm 1 with every step keeping its diagonal row, so
 * that the checked re-factorization kernel can compute it): in step
 * numbering, column k holds its U rows ascending, then k, then its L rows
 * ascending, L and U^T taking the pattern of the Cholesky factor of
 * (A + A^T)(Q,Q).  That pattern contains the pattern of the LU factors of
 * A(Q,Q) without row exchanges and equals it when A is structurally
 * symmetric; the extra entries compute to exact zeros.  With LUp (n+1),
 * LUi (nnz entries) and nU (n, U entries of each column with the diagonal)
 * all non-NULL they are filled; returns nnz, or GBLU_ERR_INVALID_INPUT for
 * an invalid pattern or a Q that is not a permutation. */
int64_t gblu_symmetric_structure(int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *Q,
                                 int64_t *LUp, int32_t *LUi, int32_t *nU);
/* The same for given pivot rows: the structure that a restart or a first
 * factorization predicts after pivot exchanges (gblu_refactorize), for the
 * steps taking the original rows piv[k] (a permutation; NULL = Q, which is
 * gblu_symmetric_structure).  With B = A(piv, Q), L and U^T take the
 * pattern of the Cholesky factor of B + B^T, which contains the pattern of
 * the LU factors of B without row exchanges (a structurally zero diagonal
 * entry of B does not matter: fill follows paths through lower steps).
 * Arguments, results and errors as gblu_symmetric_structure; piv is a host
 * array. */
int64_t gblu_predicted_structure(int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *Q,
                                 const int32_t *piv, int64_t *LUp, int32_t *LUi, int32_t *nU);
/* The structure-adaptive split of one triangular factor (Section V-A), as
 * the solve setup computes it.  count_from[p] (n+1 entries, count_from[n]
 * = 0): strict entries of the trailing block [p, n); rowlen[i] (n): all
 * entries of row i.  density == 0 is the paper's rule: P0 = the largest p
 * whose trailing block holds at least frac of all entries and at least
 * min_entries.  density > 0: P0 = the start of the longest trailing block
 * whose entry density count_from[p] / ((n-p)(n-p-1)/2) stays at least
 * density, kept if it holds min_entries entries.  Rows [P0, n) are cut
 * into `slices` pieces of about equal entry counts, each at most max_piece
 * rows: cut receives P0, the inner cut rows and n (*ncut entries; room for
 * n+1 is enough).  Returns P0, n when no block qualifies (then *ncut = 0),
 * or GBLU_ERR_INVALID_INPUT. */
int32_t gblu_solve_partition(int32_t n, const int64_t *count_from, const int64_t *rowlen, double density,
                             double frac, long long min_entries, int slices, int max_piece, int32_t *cut,
                             int32_t *ncut);
/* Column elimination tree of A(:,Q) (elimination tree of (A Q)^T (A Q)),
 * parent[k] = parent step of step k or -1 (Section II-B "ETree"). */
int gblu_column_etree(int32_t n, const int32_t *Ap, const int32_t *Ai,
                      const int32_t *Q, int32_t *parent);
/* Restart set of Section IV-C: every step that is not finished (finished[k]
 * == 0) together with all its ancestors in `parent`; out[k] = 1 for members.
 * Returns the number of members. */
int64_t gblu_restart_set(int32_t n, const int32_t *parent, const uint8_t *finished,
                         uint8_t *out);
/* Levels of a column dependency DAG given as CSC of U (rows < column are the
 * dependencies; the diagonal is ignored): level[k] = 1 + max level of its
 * dependencies (Section II-B levelization).  Returns the number of levels. */
int32_t gblu_levels(int32_t n, const int64_t *Up, const int32_t *Ui, int32_t *level);

#ifdef __cplusplus
}
#endif
#endif /* GBLU_H */
