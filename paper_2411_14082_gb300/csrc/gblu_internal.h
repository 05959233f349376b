// Internal declarations shared by the host symbolic code (symbolic.cpp),
// the kernels (kernels.cu) and the entry points (capi.cu).
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "gblu.h"

namespace gblu {

// ---------------------------------------------------------------- host side
// Validated copy of the input pattern.
struct Pattern {
    int32_t n = 0;
    std::vector<int32_t> Ap, Ai;  // caller slot order
    std::vector<int32_t> Q, qinv; // column order and its inverse
    std::vector<int32_t> cetree;  // column elimination tree of A(:,Q), by step
    std::vector<int32_t> clo;     // smallest step in the cetree subtree of each step
    int32_t cetree_height = 0;
    // row-wise copy of A for the residual: Arp[n+1], Acol[nnz], Aslot[nnz]
    std::vector<int64_t> Arp;
    std::vector<int32_t> Acol, Aslot;
};

// Host vector whose resize leaves new elements of trivial types
// uninitialized: the factor-sized index arrays are written in full by host
// threads right after they are sized, so that their pages are first touched
// in parallel rather than zeroed on one thread.
template <class T>
struct NoInitAllocator : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = NoInitAllocator<U>;
    };
    NoInitAllocator() = default;
    template <class U>
    NoInitAllocator(const NoInitAllocator<U> &) noexcept {}
    template <class U>
    void construct(U *p) noexcept
    {
        ::new ((void *)p) U;
    }
    template <class U, class... Args>
    void construct(U *p, Args &&...args)
    {
        ::new ((void *)p) U(std::forward<Args>(args)...);
    }
};
template <class T>
using BigVec = std::vector<T, NoInitAllocator<T>>;

// Fixed-pattern factor structure in step numbering (CSC, per column: the U
// rows ascending with the diagonal last, then the L rows ascending).
struct Structure {
    int32_t n = 0;
    std::vector<int64_t> LUp;  // n+1
    BigVec<int32_t> LUi;       // step numbers
    std::vector<int32_t> nU;   // U entries of each column incl. the diagonal
    std::vector<int32_t> piv;  // original row pivotal at each step
    std::vector<int32_t> pinv;
    // a predicted structure (symmetric_structure): L and U^T have the
    // pattern of one Cholesky factor
    bool symmetric = false;
    int64_t nnz() const { return LUp.empty() ? 0 : LUp.back(); }
};

// Everything derived from a Structure that the kernels use.
struct Schedule {
    // refactor: EGraph levels (Section II-B) and dual-mode split
    std::vector<int32_t> level_ptr;   // n_levels+1
    std::vector<int32_t> level_cols;  // columns sorted by level
    int32_t n_levels = 0;
    int32_t div_level = 0;            // levels [div_level, n_levels) run sync-free
    // refactor tasks: task t = task_cols[task_ptr[t] .. task_ptr[t+1]), either
    // one long column (whole CTA) or up to 8 short columns (one per warp);
    // tasks of level l < div_level are [level_task_ptr[l], level_task_ptr[l+1]),
    // the sync-free tasks start at level_task_ptr[div_level]
    std::vector<int32_t> task_ptr, task_cols, level_task_ptr;
    std::vector<int32_t> amap;        // A slot -> position inside its column
    BigVec<int32_t> LUi_orig;         // L entries: original row ids (U: step ids)
    // chain[j] = 1 iff L(:,j) = {j+1} followed by the rows of L(:,j+1), i.e.
    // j and j+1 are consecutive columns of one supernode of L
    std::vector<uint8_t> chain;
    double flops = 0;
    // solves: row-wise (CSR) copies, slots into the factor value array
    std::vector<int64_t> Lrp, Urp;        // n+1
    BigVec<int32_t> Lcol, Urow_col;       // column (step) of each entry
    BigVec<int32_t> Lslot, Uslot;         // slot in LUx
    std::vector<int32_t> Udiag;           // slot of U(i,i)
    // sparse part of each solve (rows [0, lp0) forward, [0, up0) backward),
    // solved in row blocks: block b is rows [lbs[b], lbs[b+1]), at most
    // kSolveBlockRows consecutive rows whose diagonal block is dense (rows of
    // one supernode of L forward, of U backward); lrb[i] is the block of row
    // i.  lsv_rows holds the block ids level by level (lsv_ptr), lsv_tick the
    // rows in the same order (lsv_tptr; inside a block ascending forward,
    // descending backward, so the row that finishes a block comes last);
    // lsv_div is the first sync-free level
    std::vector<int32_t> lbs, ubs, lrb, urb;
    std::vector<int32_t> lsv_ptr, lsv_rows, lsv_tptr, lsv_tick; int32_t lsv_levels = 0, lsv_div = 0;
    std::vector<int32_t> usv_ptr, usv_rows, usv_tptr, usv_tick; int32_t usv_levels = 0, usv_div = 0;
    // structure-adaptive solve (Section V): rows [p0, n) form the trailing
    // block; cut[0] = p0 < ... < cut[m] = n are the paper's slices of equal
    // entry counts (reported; the kernels use 32-row slices).  The block is
    // solved in slices of kTrailRows rows (block I = rows p0 + 32 I ...):
    // forward: row i >= lp0 has its entries before the block in CSR
    // [Lrp[i], ltri0[i - lp0]); lseg[(j - lp0) * (lnb + 1) + I] = number of
    // L entries of column j >= lp0 with row < lp0 + 32 I.
    // backward: useg[(j - up0) * (unb + 1) + I] = position (from LUp[j]) of
    // the first U entry of column j >= up0 with row >= up0 + 32 I (I = unb:
    // past the diagonal); row i < up0 has its entries in the block's
    // columns in CSR [ufar[i], Urp[i+1]).
    int32_t lp0 = 0, up0 = 0;
    int32_t lnb = 0, unb = 0;
    std::vector<int64_t> ltri0, ufar;
    BigVec<int32_t> lseg, useg;
    // dense tail of the re-factorization: columns [dense_p, n) form a
    // structurally dense block of dense_m = n - dense_p rows (0: none);
    // dense_s0[c] = slot of row dense_p inside column dense_p + c
    int32_t dense_p = 0, dense_m = 0;
    std::vector<int32_t> dense_s0;
    std::vector<int32_t> lcut, ucut;
    // columns computed row by row over their first dependencies (wide
    // columns: many dependencies in short supernode runs and a short L
    // part): pull_start[k] = how many of column k's U entries above the
    // diagonal are taken that way (0: none); pull_cols = columns with > 0
    std::vector<int32_t> pull_start;
    int64_t pull_cols = 0;
    // dividing threshold of the levels (alpha x resident warps); which parts
    // are built: the row-wise copies, and the whole solve part
    double thr = 0.0;
    bool rowwise_ready = false, solve_ready = false;
};
// wide columns: at most kPullMaxL entries in L and at least kPullMinRuns
// supernode runs among the dependencies
constexpr int kPullMaxL = 64;
constexpr int kPullMinRuns = 256;
constexpr size_t kPullScratchBytes = (size_t)1 << 30;

struct SolveSplit {
    double density = 0.0;   // > 0: longest trailing block at least this dense
    double frac = 0.7;
    long long min_entries = 300000;
    int slices = 8;
    int max_piece = 8192;   // rows of one triangular piece (shared memory)
};

// record a one-line message for gblu_last_error() and return code
int record_error(int code, const char *msg);

int validate_pattern(int32_t n, const int32_t *Ap, const int32_t *Ai, std::string &err);
void column_etree(const Pattern &P, std::vector<int32_t> &parent);
// minimum degree on A + A^T; with `group`, constrained: groups are
// eliminated in increasing order; deficiency: least estimated fill instead
// of least degree
void mindeg_order(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm,
                  const int32_t *group = nullptr, bool deficiency = false);
// multilevel nested dissection (nd_order.cpp); sets of at most `leaf`
// vertices are ordered by minimum degree, each on its own, and separators
// keep their vertex order.  constrained: the dissection only assigns groups
// (each leaf set, then each separator after its two halves) and constrained
// minimum degree orders the whole graph
void nd_order(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm, int32_t leaf,
              bool constrained = false);
// the order of fewest factorization flops among the candidate methods
// (computed on host threads); returns the GBLU_ORDER_* method chosen
int auto_order(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm);
// nnz of the Cholesky factor of (A + A^T)(Q,Q) (strict lower part), the
// size of the LU factors when every diagonal pivot is kept on a structurally
// symmetric matrix; used to size the first factorization's pool
int64_t symmetric_fill(const Pattern &P, double *flops = nullptr);
// factor structure when every step keeps its diagonal row: L and U^T with
// the pattern of that Cholesky factor (a superset of the exact LU pattern,
// equal on structurally symmetric matrices); piv = Q.  With piv given, the
// same for the steps taking the rows piv[k]: the pattern of the Cholesky
// factor of B + B^T, B = A(piv, Q), which holds the factors of B without
// row exchanges
void symmetric_structure(const Pattern &P, Structure &S, const std::vector<int32_t> *piv = nullptr);
// off-diagonal entries of A whose transposed position is not an entry of A
int64_t unsymmetric_entries(const Pattern &P);
// The schedule of a structure; with defer_solve, only what the
// re-factorization reads (the solve part follows by build_solve_schedule)
void build_schedule(const Pattern &P, const Structure &S, double alpha,
                    int resident_warps, int sched_mode, int cap_short, const SolveSplit &split,
                    int dense_min_rows, Schedule &W, bool defer_solve = false);
void build_solve_schedule(const Structure &S, const SolveSplit &split, Schedule &W);
// levels of the column dependency graph; with cut < n, the dependencies of
// columns k >= cut on columns >= cut are left out
int32_t levels_of(int32_t n, const int64_t *Up, const int32_t *Ui,
                  const int32_t *nU, std::vector<int32_t> &level, int32_t cut = INT32_MAX);

// ---------------------------------------------------------------- device side
// Control block in device memory (one per handle).
struct DevCtl {
    int32_t epoch;        // refactor epoch stored in finish[] on completion
    int32_t ticket;       // sync-free ticket counter
    int32_t interrupted;  // a pivot failed the check (Algorithms 3/4)
    int32_t first_bad;    // smallest failing column
    int32_t status;       // first error code (GBLU_ERR_*), 0 = none
    int32_t solve_epoch;  // epoch of the solve ready flags
    int32_t ticket_l, ticket_u;
    int32_t tail_epoch;   // epoch of the tail factorization done flags
    int32_t tail_ticket;
    int32_t abort_tail;   // singular / overflow seen by the tail kernel
    int32_t tail_frontier; // every step below it is final in this tail run
    unsigned long long pool_top;  // next free slot of the tail pool
    int32_t where;        // diagnostic: which wait timed out
    int32_t where_k;
    int32_t tail_mispredict;  // speculative tail: smallest step whose pivot left its preferred row
    int32_t ticket_tl, ticket_tu;  // tickets of the trailing-block solve kernels
};

#define GBLU_INTERNAL_POOL_FULL (-100)

// one ticket of a batch over sets of different patterns: task `task` of set `set`
struct SetTask {
    int32_t set, task;
};

// R: the value type of the factors being computed (double; float for the
// single-precision factorization of the mixed-precision solve)
template <typename R>
struct RefactorArgsT {
    const int32_t *Ap, *Q, *amap;   // A pattern (column pointers), order, slot map
    const double *Ax;               // new values (caller slot order)
    const int64_t *LUp;
    const int32_t *LUi, *nU;
    const uint8_t *chain;           // supernode links of L (Schedule::chain)
    // dense tail: columns k >= dense_p apply only their dependencies < dense_p
    // and leave rows >= dense_p in column k - dense_p of S (leading dim dense_ld)
    int32_t dense_p;
    const int32_t *dense_s0;
    R *S;
    int64_t dense_ld;
    R *LUx;
    int32_t *finish;
    const int32_t *task_ptr, *task_cols;
    int32_t task_begin, ntasks;     // tasks of this launch
    int32_t cap_short, cap_long;    // shared-memory work vector entries (warp / CTA)
    double eps;
    int32_t force_col = -1;         // evaluation aid: this column's check fails
    int32_t skip_done = 0;          // 1: a column whose ready flag holds the epoch is final; skip it
    // restart by re-prediction: strict_col[k] = 1 where step k's predicted
    // row is not its preferred one, so that the threshold rule takes the
    // candidate of largest magnitude there and the check asks the predicted
    // row's |x| to exceed every other candidate's; no_stop = 1: a failed
    // check records first_bad, stores the column unnormalized and publishes
    // it, and the launch runs on (later columns are then meaningless)
    const uint8_t *strict_col = nullptr;
    int32_t no_stop = 0;
    long long spin_limit;
    DevCtl *ctl;
    // wide columns (Schedule::pull_start): their first pull_start[k]
    // dependencies are applied row by row, through rows of L (CSR Lrp,
    // Lcol, Lslot) and one of pull_slots dense scratches of n values and n
    // tags (pull_lock[s] = 1 while a CTA holds scratch s); none when
    // pull_start is null
    const int32_t *pull_start = nullptr;
    const int64_t *Lrp = nullptr;
    const int32_t *Lcol = nullptr, *Lslot = nullptr;
    double *pull_x = nullptr;
    unsigned long long *pull_tag = nullptr, *pull_ctr = nullptr;
    int32_t *pull_lock = nullptr;
    int32_t pull_slots = 0, n = 0;
};
using RefactorArgs = RefactorArgsT<double>;

struct TailArgs {
    int32_t n;
    const int32_t *Ap, *Ai, *Q, *qinv;
    const double *Ax;
    const int32_t *seq;             // restart steps, ascending
    int32_t nseq;
    const int32_t *prefer;          // preferred original row per step
    const int32_t *prefer_inv;      // inverse of prefer (row -> step that preferred it)
    const int32_t *clo;             // cetree subtree lower bound per step
    int32_t *pinv;                  // original row -> step (-1 = not pivotal)
    int32_t *piv;                   // step -> original row
    int32_t *done;                  // == tail_epoch when the step is final
    // per-step column storage: entries [beg, beg+nu) are U (step ids, diagonal
    // last) and [beg+nu, beg+nu+nl) are L (original row ids)
    int64_t *cbeg;
    int32_t *cnu, *cnl;
    int32_t *rows;                  // canonical region: LUi_orig; pool after it
    double *vals;                   // canonical region: LUx; pool after it
    unsigned long long pool_base, pool_end;
    // per-CTA scratch
    double *sx;
    int32_t *smark, *slist, *sclass;
    unsigned *sbits;                // per-CTA step bitmap when it does not fit in shared memory
    int32_t bits_in_smem;           // 1: the bitmap is the kernel's dynamic shared memory
    int32_t speculate;              // 1: do not wait for an unfinished step whose preferred row is
                                    //    not in the structure (validated by tail_mispredict)
    double eps;
    long long spin_limit;
    DevCtl *ctl;
};

struct SolveArgs {
    int32_t n;
    const double *LUx;
    const int64_t *Lrp, *Urp;
    const int32_t *Lcol, *Lslot, *Ucol, *Uslot, *Udiag;
    const int32_t *piv, *Q;
    const double *b;
    double *y, *z, *x;              // forward result, backward result, output
    const int32_t *bs;              // row blocks: block b is rows [bs[b], bs[b+1])
    const int32_t *rb;              // block of each row
    double *ext;                    // per row: its sum over entries outside its block
    double *far;                    // backward, rows < up0: their sum over the trailing block's columns
    const int64_t *ufar;            // backward, rows < up0: first CSR entry in those columns (null: none)
    const int32_t *rows;            // rows in ticket order, or block ids (level finish)
    int32_t nrows;                  // number of entries of rows
    // batches (nsets > 1): set s reads LUx + s*lu_stride, b + s*b_stride and
    // writes x + s*x_stride; y, z and ext are per set at s*v_stride
    int32_t nsets;
    int64_t lu_stride, b_stride, x_stride, v_stride;
    long long spin_limit;
    DevCtl *ctl;
};

// kernel launchers (kernels.cu); each returns a cudaError_t as int
int launch_begin_refactor(DevCtl *ctl, void *stream);
int refactor_setup(int cap_long, int *blocks_per_sm, int *batch_blocks_per_sm);
int refactor_setup_f32(int cap_long, int *blocks_per_sm);
int launch_refactor_tasks(const RefactorArgs &a, bool pipeline, int grid, int epoch, void *stream);
// the same tasks with single-precision factor values (no dense tail)
int launch_refactor_tasks_f32(const RefactorArgsT<float> &a, bool pipeline, int grid, int epoch, void *stream);
// batch of value sets on one structure (sets_dev: one argument block per set)
int launch_begin_batch(DevCtl *ctl, int nsets, int32_t *ticket, void *stream);
int launch_refactor_batch(const RefactorArgs *sets_dev, const RefactorArgs &a0, int nsets, bool pipeline,
                          int grid, int epoch, int32_t *ticket, void *stream, int group);
int launch_refactor_multi(const RefactorArgs *sets_dev, const RefactorArgs &a0, int nsets, const SetTask *order_dev,
                          int npairs, int grid, int epoch, int32_t *ticket, void *stream, bool pull);
int launch_begin_tail(DevCtl *ctl, unsigned long long pool_base, void *stream);
int launch_tail_init(int32_t n, const int32_t *restart_mask, const int32_t *piv_old,
                     int32_t *pinv, int32_t *piv, int32_t *done, int epoch, void *stream);
int launch_tail(const TailArgs &a, int grid, int epoch, void *stream);
// another speculative pass over the steps seq[0..nseq): their pivots, row
// map entries and done flags are cleared; the pool and the other steps stay
int launch_tail_repass(DevCtl *ctl, const int32_t *seq, int32_t nseq, int32_t n, int32_t *piv, int32_t *pinv,
                       int32_t *done, void *stream);
int tail_setup();
constexpr int32_t kTailSmemBits = 1 << 19;   // steps whose bitmap fits in shared memory
int launch_pool_scatter(const int32_t *seq, int32_t nseq, const int64_t *cbeg, const int32_t *cnu,
                        const int32_t *cnl, const int32_t *prow, const int64_t *LUp, const int32_t *LUi,
                        const int32_t *pinv, int32_t n, double *vals, int32_t *bad, void *stream);
// the pivot of step k after its check failed: the candidate of largest |x|
// in column k (values unnormalized), out[0] its step, out[1] a non-finite flag
int launch_pivot_choice(const int64_t *LUp, const int32_t *LUi, const double *LUx, const int32_t *nU,
                        const int32_t *piv, const int32_t *qinv, int32_t k, int32_t *out, void *stream);
// dense tail of the re-factorization (dense.cu)
struct DenseArgs2 {
    double *S;                      // m x m, column-major, leading dimension ld
    int64_t ld;
    int32_t m, p;                   // block rows, first column of the block
    double eps;
    DevCtl *ctl;
    const int64_t *LUp;
    const int32_t *s0;              // slot of row p inside column p + c
    double *LUx;
    int32_t *finish;
    int epoch;
};
constexpr int kDenseNb = 8;         // panel width
int dense_setup(int max_rows);
int launch_dense_lu(const DenseArgs2 &d, void *stream, long long *launches);

int launch_gather_scale(int64_t m, const int32_t *src, const double *scale, const double *in, double *out,
                        void *stream);
int launch_widen(const float *src, double *dst, int64_t n, void *stream);
// double-precision verification of single-precision pivots: a column whose
// pivot does not clear the threshold by the single-precision error estimate
// sets interrupted / first_bad
int launch_f32_verify(int32_t n, const int64_t *LUp, const int32_t *LUi, const int32_t *nU, const float *LUx,
                      const int64_t *Lrp, const int32_t *Lcol, const int32_t *Lslot, double eps, DevCtl *ctl,
                      int grid, void *stream);
int launch_axpy(double *x, const double *d, int32_t n, void *stream);
int launch_begin_solve(DevCtl *ctl, double *y, double *z, double *el, double *eu, int n, void *stream);
int launch_solve_finish(const SolveArgs &a, bool lower, void *stream);
int launch_lsolve(const SolveArgs &a, bool level_mode, int grid, void *stream);
int launch_usolve(const SolveArgs &a, bool level_mode, int grid, void *stream);
// several handles' sparse solves in one launch per triangle (no dense pieces)
int launch_solve_multi(const SolveArgs *lo, const SolveArgs *up, int nsets, int max_n, const SetTask *order_l,
                       int total_l, const SetTask *order_u, int total_u, int grid, int32_t *tickets, void *stream);
int launch_residual(int32_t n, const int64_t *Arp, const int32_t *Acol,
                    const int32_t *Aslot, const double *Ax, const double *b,
                    const double *x, double *out, double *partial, int nblocks,
                    void *stream, double *rvec = nullptr);
int solve_syncfree_grid(int *grid);
// one trapezoid slice of the trailing block: rectangular part, then triangular piece
// trailing block of the structure-adaptive solve, rows [p0, n) in slices of
// kTrailRows rows.  Forward: the rows' sums over the columns before p0
// (into ext), then the slices, sync-free; backward: the slices, then the
// sums of rows < p0 over the block's columns (into far)
struct TrailArgs {
    int32_t p0, n, nb;
    const int32_t *seg;             // lseg / useg of the Schedule
    const int64_t *LUp;
    const int32_t *LUi, *nU;
    const int64_t *rows;            // forward: ltri0; backward: ufar
};
int launch_trail(const SolveArgs &a, const TrailArgs &t, bool lower, int grid, void *stream);
int trail_setup(int *blocks_per_sm);

constexpr int kRefThreads = 256;       // 8 warps per refactor CTA
constexpr int kRefCapShort = 640;      // work-vector entries per warp (short columns)
constexpr int kRefCapLong = 8 * kRefCapShort;  // per CTA (long columns), 60 KB: 3 CTAs per SM
constexpr int kTailThreads = 256;
constexpr int kSolveWarpsPerBlock = 8;
constexpr int kSolveBlockRows = 32;   // rows of one block of the sparse solves
constexpr int kSolveBlockThreads = 256;
constexpr int kMaxPieceRows = 4096;    // rows of one paper slice (reported partition)
constexpr int kTrailRows = 32;         // rows of one slice of the trailing-block kernels

}  // namespace gblu
