// C-ABI entry points of libgblu: handle management, analyze, factorize,
// checked re-factorization with restart, solve, residual, stats and export.
// The orchestration runs on the host; every numerical step runs in the
// kernels of kernels.cu.
#include <queue>
#include <atomic>
#include <thread>
#include <nvtx3/nvToolsExt.h>
#include <chrono>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "gblu_internal.h"

using namespace gblu;

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? GBLU_ERR_NOMEM : GBLU_ERR_CUDA, \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                        \
    } while (0)

#define CK(call)                                   \
    do {                                           \
        int r_ = (call);                           \
        if (r_ != 0) return r_;                    \
    } while (0)

#define KL(call)                                                                        \
    do {                                                                                \
        h->launches++;                                                                  \
        int e_ = (call);                                                                \
        if (e_ != 0)                                                                    \
            return fail(GBLU_ERR_CUDA, "kernel launch %s failed: %s", #call,            \
                        cudaGetErrorString((cudaError_t)e_));                            \
    } while (0)

// Device buffer with capacity tracking.
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t cap = 0;  // elements
};

}  // namespace

int gblu::record_error(int code, const char *msg)
{
    g_err = msg;
    return code;
}

struct gblu_ctx {
    int device = 0;
    gblu_opts opts{};
    int sm_count = 0;
    int l2_bytes = 0;
    int ref_blocks_per_sm = 0, ref_grid = 0, solve_grid = 0, res_blocks = 0, trail_per_sm = 0;
    int batch_blocks_per_sm = 0;   // refactor_batch_kernel CTAs that fit on an SM
    int ref32_blocks_per_sm = 0, ref32_grid = 0;
    bool f32_valid = false, f32_widened = false;   // single-precision factors of the last call
    int32_t force_col = -1;                        // forced check failure of the next refactorization
    double t_tail[4] = {0, 0, 0, 0};               // last tail run: kernel, repack, schedule, upload (ms)
    int32_t tail_passes = 0;                       // kernel passes of the last tail run
    int32_t first_mode = 0;                        // last gblu_factorize: 0 pivoting kernel only,
                                                   // 1 predicted structure, 2 and then the pivoting kernel
    double t_first_symbolic = 0.0;                 // its structure prediction (host ms)
    bool predicted = false;                        // the installed structure is a symmetric prediction
    int32_t repredictions = 0;                     // structure re-predictions of the last restart or
                                                   // first factorization
    bool strict_on = false, no_stop = false;       // re-factorization check modes of a re-prediction
    bool solve_pending = false;                    // an install's solve part is still to be built
    bool last_repivot = false;                     // the last refactorization restarted
    bool analyzed = false, factorized = false;
    Pattern P;
    Structure S;
    Schedule W;
    int32_t epoch = 0, tail_epoch = 0;
    int64_t n_refactor = 0, n_repivot = 0, n_restart_cols = 0;
    int64_t launches = 0;
    int32_t last_first_bad = -1;
    size_t device_bytes = 0;
    DevCtl *hctl = nullptr;  // pinned mirror
    DevCtl *ctl = nullptr;
    // pattern / order
    DBuf<int32_t> Ap, Ai, Q, qinv, clo, Acol, Aslot;
    DBuf<int64_t> Arp;
    // factor structure and values: rows/vals hold the canonical columns
    // followed by the restart pool
    DBuf<int64_t> LUp;
    DBuf<int32_t> LUi, nU, rows, finish, task_ptr, task_cols, amap, piv, pinv;
    DBuf<uint8_t> chain;
    // re-prediction: steps whose predicted row is not the preferred one, and
    // the pivot choice read back (step, non-finite flag)
    DBuf<uint8_t> strict;
    DBuf<int32_t> pchoice;
    // wide columns taken row by row: their pull starts and the per-CTA dense
    // scratch (pull_slots CTAs x n values and n tags, one counter each)
    DBuf<int32_t> pull_start;
    DBuf<double> pull_x;
    DBuf<unsigned long long> pull_tag, pull_ctr;
    DBuf<int32_t> pull_lock;
    int32_t pull_slots = 0;
    DBuf<double> vals;
    // solves
    DBuf<int64_t> Lrp, Urp;
    DBuf<int32_t> Lcol, Lslot, Ucol, Uslot, Udiag, lsv_rows, usv_rows, lbs, ubs, lrb, urb, lsv_tick, usv_tick,
        lseg, useg;
    DBuf<int64_t> ltri0, ufar;
    DBuf<double> y, z, ext_l, ext_u, far, partial, stage_ax, stage_b, stage_x;
    // dense tail of the re-factorization: the block and its column offsets
    DBuf<double> dense;
    DBuf<int32_t> dense_s0;
    // batches of value sets: ready flags and control blocks per set, the
    // argument blocks, the ticket
    DBuf<int32_t> bfinish, bticket;
    DBuf<DevCtl> bctl;
    DBuf<RefactorArgs> bargs;
    // mixed precision: single-precision factors, their widened copy, the
    // residual and correction vectors, and the residual norms (host mirror)
    DBuf<float> vals32;
    DBuf<double> vals_w, ir_r, ir_d, ir_out;
    double *ir_host = nullptr;
    std::vector<RefactorArgs> bargs_host;
    std::vector<DevCtl> bctl_host;
    // restart (tail factorization)
    DBuf<int32_t> seq, restart, done, tpiv, tpinv, cnu, cnl, smark, slist, sclass;
    DBuf<int64_t> cbeg;
    DBuf<int32_t> sflag;
    DBuf<unsigned> sbits;
    // multi-pattern batches led by this handle: merged ticket order, cached
    // for the handles (and structure versions) it was built for
    DBuf<SetTask> morder;
    std::vector<std::pair<const void *, uint64_t>> morder_key;
    int64_t morder_n = 0;
    DBuf<SetTask> mlorder, muorder;   // merged row tickets of multi-pattern solves
    std::vector<std::pair<const void *, uint64_t>> msolve_key;
    int64_t mlorder_n = 0, muorder_n = 0;
    DBuf<SolveArgs> margs;
    std::vector<SolveArgs> margs_host;
    DBuf<int32_t> mticket;
    // captured refactor + solve (gblu_step): replayed while the structure is
    // the one it was captured on
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    cudaStream_t aux = nullptr;      // this handle's solves forked off a multi-pattern call
    uint64_t gversion = 0;
    int32_t *epoch_host = nullptr;   // pinned: the epoch the next replay stores
    long long glaunches = 0;         // kernels per replay
    uint64_t struct_version = 0;
    uint64_t layout_version = 0;     // bumped by every device (re)allocation
    uint64_t glayout = 0;
    // captured batch refactor + batch solve (gblu_step_batch): replayed while
    // the structure, the device layout and the caller's buffers are the ones
    // it was captured with
    cudaGraphExec_t bgexec = nullptr;
    std::vector<int64_t> bgkey;      // nsets, buffer addresses and strides
    uint64_t bgversion = 0, bglayout = 0;
    long long bglaunches = 0;
    DBuf<RefactorArgs> bgargs;       // argument blocks the graph reads
    DevCtl *bgctl_host = nullptr;    // pinned: per-set control blocks after a replay
    int32_t bgctl_cap = 0;
    DBuf<double> sx;
};

namespace {

// a first factorization (whose pivot prediction, the diagonal, has no
// history behind it) speculates while at most this many steps of a pass
// leave their diagonal rows
constexpr int kSpecMaxMoved = 4;

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// an NVTX range over one library call, for profilers (no cost without one)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// events of one call, destroyed on every way out of it (an event whose
// work is still pending is released once that work completes)
struct EventList {
    std::vector<cudaEvent_t> ev;
    EventList() = default;
    EventList(const EventList &) = delete;
    EventList &operator=(const EventList &) = delete;
    ~EventList()
    {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    int record(cudaStream_t s, cudaEvent_t *out)
    {
        cudaEvent_t e;
        CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ev.push_back(e);
        CU(cudaEventRecord(e, s));
        *out = e;
        return GBLU_OK;
    }
};

// SMs the handle's persistent launches may use (the max_sms option), and a
// persistent grid of per_sm CTAs on each of them
int sms_used(const gblu_ctx *h)
{
    return (h->opts.max_sms > 0 && h->opts.max_sms < h->sm_count) ? h->opts.max_sms : h->sm_count;
}
int pgrid(const gblu_ctx *h, int per_sm) { return std::max(1, per_sm) * sms_used(h); }

template <class T>
int ensure(gblu_ctx *h, DBuf<T> &b, size_t count)
{
    if (count == 0) count = 1;
    if (b.cap >= count) return GBLU_OK;
    if (b.p) {
        cudaFree(b.p);
        h->device_bytes -= b.cap * sizeof(T);
        b.p = nullptr;
        b.cap = 0;
    }
    h->layout_version++;   // captured graphs hold the old address
    cudaError_t e = cudaMalloc((void **)&b.p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GBLU_ERR_NOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                    cudaGetErrorString(e));
    }
    b.cap = count;
    h->device_bytes += count * sizeof(T);
    return GBLU_OK;
}

template <class T>
void release(gblu_ctx *h, DBuf<T> &b)
{
    if (b.p) {
        cudaFree(b.p);
        h->device_bytes -= b.cap * sizeof(T);
        h->layout_version++;
    }
    b.p = nullptr;
    b.cap = 0;
}

template <class T, class A>
int upload(gblu_ctx *h, DBuf<T> &b, const std::vector<T, A> &v, cudaStream_t st)
{
    CK(ensure(h, b, v.size()));
    if (!v.empty()) CU(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return GBLU_OK;
}

int read_ctl(gblu_ctx *h, cudaStream_t st)
{
    CU(cudaMemcpyAsync(h->hctl, h->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return GBLU_OK;
}

int status_code(gblu_ctx *h)
{
    const int s = h->hctl->status;
    if (s == 0) return GBLU_OK;
    if (s == GBLU_ERR_DEVICE_TIMEOUT)
        return fail(s, "device wait timed out (site %d, column %d)", h->hctl->where, h->hctl->where_k);
    if (s == GBLU_ERR_SINGULAR) return fail(s, "singular: no nonzero pivot candidate at step %d", h->hctl->where_k);
    if (s == GBLU_ERR_INTERNAL) return fail(s, "internal structure check failed on the device");
    if (s == GBLU_ERR_NONFINITE)
        return fail(s, "a NaN or infinite value in the column of step %d (check the values of A)", h->hctl->where_k);
    return fail(s, "device status %d", s);
}

static SolveSplit solve_split(const gblu_opts &o)
{
    SolveSplit sp;
    sp.density = o.solve_dense_density;
    sp.frac = o.solve_dense_frac;
    sp.min_entries = o.solve_dense_min;
    sp.slices = o.solve_slices;
    sp.max_piece = kMaxPieceRows;
    return sp;
}

// The solve part of the schedule on the device (and the original row ids of
// the restart kernel); l_rows_done: the row-wise copy of L went up with the
// re-factorization part (the wide columns read it).  Synchronizes `st`:
// the host vectors are uploaded asynchronously.
static int upload_solve(gblu_ctx *h, cudaStream_t st, bool l_rows_done)
{
    const int32_t n = h->S.n;
    const size_t nnz = (size_t)h->S.nnz();
    if (nnz > 0)
        CU(cudaMemcpyAsync(h->rows.p, h->W.LUi_orig.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (!l_rows_done) {
        CK(upload(h, h->Lrp, h->W.Lrp, st));
        CK(upload(h, h->Lcol, h->W.Lcol, st));
        CK(upload(h, h->Lslot, h->W.Lslot, st));
    }
    CK(upload(h, h->Urp, h->W.Urp, st));
    CK(upload(h, h->Ucol, h->W.Urow_col, st));
    CK(upload(h, h->Uslot, h->W.Uslot, st));
    CK(upload(h, h->Udiag, h->W.Udiag, st));
    CK(upload(h, h->lsv_rows, h->W.lsv_rows, st));
    CK(upload(h, h->usv_rows, h->W.usv_rows, st));
    CK(upload(h, h->lbs, h->W.lbs, st));
    CK(upload(h, h->ubs, h->W.ubs, st));
    CK(upload(h, h->lrb, h->W.lrb, st));
    CK(upload(h, h->urb, h->W.urb, st));
    CK(upload(h, h->lsv_tick, h->W.lsv_tick, st));
    CK(upload(h, h->usv_tick, h->W.usv_tick, st));
    CK(upload(h, h->ltri0, h->W.ltri0, st));
    CK(upload(h, h->lseg, h->W.lseg, st));
    CK(upload(h, h->ufar, h->W.ufar, st));
    CK(upload(h, h->useg, h->W.useg, st));
    if (h->W.up0 < n) CK(ensure(h, h->far, (size_t)n));
    CU(cudaStreamSynchronize(st));
    return GBLU_OK;
}

// Install a factor structure: schedule on the host, arrays on the device.
// values (optional) are the factor values in canonical order.  With
// defer_solve only what the re-factorization reads is built and uploaded
// (nothing synchronizes); finish_install adds the rest, on the host while
// the stream runs the re-factorization.
int install_structure(gblu_ctx *h, Structure &&S, const std::vector<double> *values, cudaStream_t st,
                      bool defer_solve = false)
{
    h->S = std::move(S);
    h->struct_version++;
    h->f32_valid = false;
    const int resident_warps = h->ref_blocks_per_sm * h->sm_count * (kRefThreads / 32);
    const SolveSplit sp = solve_split(h->opts);
    const auto t_s = std::chrono::steady_clock::now();
    build_schedule(h->P, h->S, h->opts.alpha, resident_warps, h->opts.sched_mode, h->opts.warp_column_max, sp,
                   h->opts.dense_min_rows, h->W, defer_solve);
    h->solve_pending = defer_solve;
    const auto t_u = std::chrono::steady_clock::now();
    h->t_tail[2] = std::chrono::duration<double, std::milli>(t_u - t_s).count();
    for (int32_t v : h->W.amap)
        if (v < 0) return fail(GBLU_ERR_INTERNAL, "an entry of A is outside the factor pattern");
    const int32_t n = h->S.n;
    const size_t nnz = (size_t)h->S.nnz();
    CK(upload(h, h->LUp, h->S.LUp, st));
    CK(upload(h, h->LUi, h->S.LUi, st));
    CK(upload(h, h->nU, h->S.nU, st));
    CK(upload(h, h->chain, h->W.chain, st));
    h->pull_slots = 0;
    if (h->W.pull_cols > 0) {
        // one scratch per CTA that a persistent launch can hold; only while it
        // stays within kPullScratchBytes (the columns are pushed otherwise)
        const int slots = std::max(h->ref_blocks_per_sm, h->batch_blocks_per_sm) * h->sm_count;
        const size_t bytes = (size_t)slots * (size_t)n * (sizeof(double) + sizeof(unsigned long long));
        if (bytes <= kPullScratchBytes) {
            CK(upload(h, h->pull_start, h->W.pull_start, st));
            CK(ensure(h, h->pull_x, (size_t)slots * n));
            CK(ensure(h, h->pull_tag, (size_t)slots * n));
            CK(ensure(h, h->pull_ctr, (size_t)slots));
            CK(ensure(h, h->pull_lock, (size_t)slots));
            // tags start below every counter value; every scratch free
            CU(cudaMemsetAsync(h->pull_tag.p, 0, sizeof(unsigned long long) * (size_t)slots * n, st));
            CU(cudaMemsetAsync(h->pull_ctr.p, 0, sizeof(unsigned long long) * (size_t)slots, st));
            CU(cudaMemsetAsync(h->pull_lock.p, 0, sizeof(int32_t) * (size_t)slots, st));
            h->pull_slots = slots;
        }
    }
    CK(upload(h, h->dense_s0, h->W.dense_s0, st));
    if (h->W.dense_m > 0) CK(ensure(h, h->dense, (size_t)h->W.dense_m * h->W.dense_m));
    CK(upload(h, h->piv, h->S.piv, st));
    CK(upload(h, h->pinv, h->S.pinv, st));
    CK(upload(h, h->task_ptr, h->W.task_ptr, st));
    CK(upload(h, h->task_cols, h->W.task_cols, st));
    CK(upload(h, h->amap, h->W.amap, st));
    CK(ensure(h, h->finish, n));
    CK(ensure(h, h->y, n));
    CK(ensure(h, h->z, n));
    CK(ensure(h, h->ext_l, n));
    CK(ensure(h, h->ext_u, n));
    // ready flags hold epochs (> 0); recycled device memory may hold any
    // value, so they start from zero
    CU(cudaMemsetAsync(h->finish.p, 0, sizeof(int32_t) * n, st));
    // canonical rows/vals; the pool is sized at restart time
    if (h->rows.cap < nnz || h->vals.cap < nnz) {
        CK(ensure(h, h->rows, nnz));
        CK(ensure(h, h->vals, nnz));
    }
    if (values && nnz > 0)
        CU(cudaMemcpyAsync(h->vals.p, values->data(), nnz * sizeof(double), cudaMemcpyHostToDevice, st));
    if (defer_solve) {
        // the wide columns read the rows of L; the host vectors stay alive
        // in the handle until finish_install synchronizes
        if (h->W.rowwise_ready) {
            CK(upload(h, h->Lrp, h->W.Lrp, st));
            CK(upload(h, h->Lcol, h->W.Lcol, st));
            CK(upload(h, h->Lslot, h->W.Lslot, st));
        }
        h->t_tail[3] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_u).count();
        return GBLU_OK;
    }
    CK(upload_solve(h, st, false));
    h->t_tail[3] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_u).count();
    return GBLU_OK;
}

// The solve part of a deferred install_structure: built on the host (while
// the stream may still run a re-factorization, which does not read it),
// then uploaded behind the work on the stream.
int finish_install(gblu_ctx *h, cudaStream_t st)
{
    if (!h->solve_pending) return GBLU_OK;
    const bool l_rows_done = h->W.rowwise_ready;
    const auto t_s = std::chrono::steady_clock::now();
    build_solve_schedule(h->S, solve_split(h->opts), h->W);
    h->t_tail[2] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_s).count();
    // its uploads wait behind the stream's work, so their time is the
    // caller's (the re-factorization's), not tail_upload_ms
    CK(upload_solve(h, st, l_rows_done));
    h->solve_pending = false;
    return GBLU_OK;
}

// Checked re-factorization on the installed structure (Algorithms 3 and 4).
// *interrupted = 1 if a pivot failed the check.
// argument block of the column kernels for the installed structure
RefactorArgs refactor_args(gblu_ctx *h, const double *Ax)
{
    RefactorArgs a{};
    a.Ap = h->Ap.p;
    a.Q = h->Q.p;
    a.amap = h->amap.p;
    a.Ax = Ax;
    a.LUp = h->LUp.p;
    a.LUi = h->LUi.p;
    a.nU = h->nU.p;
    a.chain = h->chain.p;
    a.dense_p = h->W.dense_m > 0 ? h->W.dense_p : INT_MAX;   // INT_MAX: no dense tail
    a.dense_s0 = h->dense_s0.p;
    a.S = h->dense.p;
    a.dense_ld = h->W.dense_m;
    a.LUx = h->vals.p;
    a.finish = h->finish.p;
    a.task_ptr = h->task_ptr.p;
    a.task_cols = h->task_cols.p;
    a.cap_short = h->opts.warp_column_max;
    a.cap_long = kRefCapLong;
    a.eps = h->opts.pivot_tol;
    a.force_col = h->force_col;
    a.spin_limit = h->opts.spin_limit;
    a.ctl = h->ctl;
    a.strict_col = h->strict_on ? h->strict.p : nullptr;
    a.no_stop = h->no_stop ? 1 : 0;
    if (h->pull_slots > 0) {
        a.pull_start = h->pull_start.p;
        a.Lrp = h->Lrp.p;
        a.Lcol = h->Lcol.p;
        a.Lslot = h->Lslot.p;
        a.pull_x = h->pull_x.p;
        a.pull_tag = h->pull_tag.p;
        a.pull_ctr = h->pull_ctr.p;
        a.pull_lock = h->pull_lock.p;
        a.pull_slots = h->pull_slots;
    }
    a.n = h->S.n;
    return a;
}

// the launches of one checked re-factorization; ep = the epoch the kernels
// store in the ready flags, or -1: read it from the control block (graph
// replay, where the epoch changes between launches of the same graph)
int issue_refactor(gblu_ctx *h, const double *Ax, cudaStream_t st, int ep)
{
    KL(launch_begin_refactor(h->ctl, st));
    RefactorArgs a = refactor_args(h, Ax);
    const std::vector<int32_t> &ltp = h->W.level_task_ptr;
    const int32_t div = h->W.div_level;   // the schedule already follows sched_mode
    for (int32_t l = 0; l < div; l++) {   // cluster mode: one launch per level
        a.task_begin = ltp[l];
        a.ntasks = ltp[l + 1] - ltp[l];
        KL(launch_refactor_tasks(a, false, 0, ep, st));
    }
    const int32_t ntask = (int32_t)h->W.task_ptr.size() - 1;
    if (ltp[div] < ntask) {               // pipeline mode: one persistent launch
        a.task_begin = ltp[div];
        a.ntasks = ntask - ltp[div];
        KL(launch_refactor_tasks(a, true, pgrid(h, h->ref_blocks_per_sm), ep, st));
    }
    if (h->W.dense_m > 0) {   // the dense tail: blocked LU of the block, then scatter
        DenseArgs2 d{};
        d.S = h->dense.p;
        d.ld = h->W.dense_m;
        d.m = h->W.dense_m;
        d.p = h->W.dense_p;
        d.eps = h->opts.pivot_tol;
        d.ctl = h->ctl;
        d.LUp = h->LUp.p;
        d.s0 = h->dense_s0.p;
        d.LUx = h->vals.p;
        d.finish = h->finish.p;
        d.epoch = ep;
        long long nl = 0;
        const int e = launch_dense_lu(d, st, &nl);
        h->launches += nl;
        if (e != 0) return fail(GBLU_ERR_CUDA, "dense tail launch failed: %s", cudaGetErrorString((cudaError_t)e));
    }
    return GBLU_OK;
}

// A deferred install's solve part is finished on the host while the
// re-factorization runs.
int run_refactor(gblu_ctx *h, const double *Ax, cudaStream_t st, int *interrupted)
{
    h->epoch++;
    CK(issue_refactor(h, Ax, st, h->epoch));
    CK(finish_install(h, st));
    CK(read_ctl(h, st));
    CK(status_code(h));
    *interrupted = h->hctl->interrupted;
    h->last_first_bad = h->hctl->interrupted ? h->hctl->first_bad : -1;
    return GBLU_OK;
}

// Factorization with threshold pivoting of the steps in rmask (Algorithm 5;
// Algorithm 1 when rmask holds every step); the other steps keep their
// current columns.  Rebuilds the structure and the schedule afterwards.
// speculate: passes predict that every step takes its preferred row;
// keep_if_same: a restart, whose structure stays when every pivot is kept.
int run_tail(gblu_ctx *h, const double *Ax, cudaStream_t st, const std::vector<uint8_t> &rmask,
             size_t pool_hint, bool keep_if_same, bool speculate)
{
    const Pattern &P = h->P;
    const int32_t n = P.n;
    const Structure &S = h->S;
    const int64_t nnz = S.nnz();
    int64_t nR = 0;
    for (uint8_t v : rmask) nR += v != 0;
    std::vector<int32_t> seq, rm(n);
    seq.reserve(nR);
    int64_t restart_len = 0;
    for (int32_t k = 0; k < n; k++) {
        rm[k] = rmask[k];
        if (rmask[k]) {
            seq.push_back(k);
            restart_len += S.LUp[k + 1] - S.LUp[k];
        }
    }
    // canonical descriptors for the columns that keep their values
    std::vector<int64_t> cbeg(n);
    std::vector<int32_t> cnu(n), cnl(n);
    for (int32_t k = 0; k < n; k++) {
        cbeg[k] = S.LUp[k];
        cnu[k] = S.nU[k];
        cnl[k] = (int32_t)(S.LUp[k + 1] - S.LUp[k]) - S.nU[k];
    }
    CK(upload(h, h->seq, seq, st));
    CK(upload(h, h->restart, rm, st));
    CK(upload(h, h->cbeg, cbeg, st));
    CK(upload(h, h->cnu, cnu, st));
    CK(upload(h, h->cnl, cnl, st));
    CK(ensure(h, h->done, n));
    CK(ensure(h, h->tpiv, n));
    CK(ensure(h, h->tpinv, n));
    // scratch: one dense work vector per CTA
    int slots = std::min<int64_t>((int64_t)nR, (int64_t)sms_used(h) * 2);
    const size_t per_slot = (size_t)n * (sizeof(double) + 2 * sizeof(int32_t));
    const size_t budget = (size_t)4 << 30;
    slots = (int)std::max<size_t>(1, std::min<size_t>((size_t)slots, budget / per_slot));
    CK(ensure(h, h->sx, (size_t)slots * n));
    CK(ensure(h, h->smark, (size_t)slots * n));
    CK(ensure(h, h->slist, (size_t)slots * n));
    CK(ensure(h, h->sclass, (size_t)slots * n));
    const bool bits_smem = n <= kTailSmemBits;
    const size_t words = ((size_t)n + 31) / 32;
    if (!bits_smem) CK(ensure(h, h->sbits, (size_t)slots * words));
    // pool after the canonical columns
    // speculative restarts may write a column once per pass
    size_t pool = std::max<size_t>(pool_hint, (size_t)std::max<int64_t>((speculate ? 4 : 2) * restart_len,
                                                                        (int64_t)P.Ai.size())) +
                  (size_t)n;
    using TClock = std::chrono::steady_clock;
    auto ms_since = [](TClock::time_point t) {
        return std::chrono::duration<double, std::milli>(TClock::now() - t).count();
    };
    CU(cudaStreamSynchronize(st));
    const TClock::time_point t_k = TClock::now();
    for (int attempt = 0; attempt < 8; attempt++) {
        const size_t need = (size_t)nnz + pool;
        if (h->rows.cap < need || h->vals.cap < need) {
            // grow, keeping the canonical region
            DBuf<int32_t> nr;
            DBuf<double> nv;
            CK(ensure(h, nr, need));
            CK(ensure(h, nv, need));
            if (nnz > 0) {
                CU(cudaMemcpyAsync(nr.p, h->rows.p, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
                CU(cudaMemcpyAsync(nv.p, h->vals.p, nnz * sizeof(double), cudaMemcpyDeviceToDevice, st));
            }
            CU(cudaStreamSynchronize(st));
            release(h, h->rows);
            release(h, h->vals);
            h->rows = nr;
            h->vals = nv;
        }
        h->tail_epoch++;
        KL(launch_begin_tail(h->ctl, (unsigned long long)nnz, st));
        KL(launch_tail_init(n, h->restart.p, h->piv.p, h->tpinv.p, h->tpiv.p, h->done.p, h->tail_epoch, st));
        CU(cudaMemsetAsync(h->smark.p, 0, (size_t)slots * n * sizeof(int32_t), st));
        if (!bits_smem) CU(cudaMemsetAsync(h->sbits.p, 0, (size_t)slots * words * sizeof(unsigned), st));
        TailArgs t{};
        t.n = n;
        t.Ap = h->Ap.p;
        t.Ai = h->Ai.p;
        t.Q = h->Q.p;
        t.qinv = h->qinv.p;
        t.Ax = Ax;
        t.seq = h->seq.p;
        t.nseq = (int32_t)nR;
        t.prefer = h->piv.p;
        t.prefer_inv = h->pinv.p;
        t.clo = h->clo.p;
        t.pinv = h->tpinv.p;
        t.piv = h->tpiv.p;
        t.done = h->done.p;
        t.cbeg = h->cbeg.p;
        t.cnu = h->cnu.p;
        t.cnl = h->cnl.p;
        t.rows = h->rows.p;
        t.vals = h->vals.p;
        t.pool_base = (unsigned long long)nnz;
        t.pool_end = (unsigned long long)(nnz + pool);
        t.sx = h->sx.p;
        t.smark = h->smark.p;
        t.slist = h->slist.p;
        t.sclass = h->sclass.p;
        t.sbits = bits_smem ? nullptr : h->sbits.p;
        t.bits_in_smem = bits_smem ? 1 : 0;
        t.eps = h->opts.pivot_tol;
        t.spin_limit = h->opts.spin_limit;
        t.ctl = h->ctl;
        // a speculative pass predicts that the steps take their preferred
        // pivots; after a pass in which some step took another row, the
        // steps after the first such step run again.  The last pass runs
        // without speculation: after kMaxSpecPasses, after a pass that
        // finished no step for good, and, in a first factorization (whose
        // prediction, the diagonal, has no pivot history behind it), after
        // a pass in which more than kSpecMaxMoved finished steps left their
        // preferred rows (each wrong prediction costs a pass; a pivot that
        // moves takes another step's row, so one miss moves two steps)
        constexpr int kMaxSpecPasses = 8;
        std::vector<int32_t> cur = seq;
        bool pool_full = false, spec = speculate;
        for (int pass = 0;; pass++) {
            t.speculate = (spec && pass < kMaxSpecPasses) ? 1 : 0;
            t.nseq = (int32_t)cur.size();
            KL(launch_tail(t, slots, h->tail_epoch, st));
            CK(read_ctl(h, st));
            h->tail_passes = pass + 1;
            if (h->hctl->status == GBLU_INTERNAL_POOL_FULL) {
                pool_full = true;
                break;
            }
            CK(status_code(h));
            if (!t.speculate || h->hctl->tail_mispredict == INT_MAX) break;
            int32_t js = h->hctl->tail_mispredict;
            // a pass stopped early (a column found its speculation broken)
            // may leave steps before js unfinished; a finished step is only
            // known right if every step before it finished, so the next pass
            // starts at the first unfinished step at the latest
            const bool count_moved = !keep_if_same;
            if (h->hctl->abort_tail || count_moved) {
                std::vector<int32_t> dn(n), tp;
                CU(cudaMemcpyAsync(dn.data(), h->done.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
                if (count_moved) {
                    tp.resize(n);
                    CU(cudaMemcpyAsync(tp.data(), h->tpiv.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
                }
                CU(cudaStreamSynchronize(st));
                if (h->hctl->abort_tail)
                    for (int32_t k : cur)
                        if (dn[k] != h->tail_epoch) {
                            js = std::min(js, k - 1);
                            break;   // cur is ascending
                        }
                if (count_moved) {
                    int64_t moved = 0;
                    for (int32_t k : cur) moved += dn[k] == h->tail_epoch && tp[k] != S.piv[k];
                    if (moved > kSpecMaxMoved) spec = false;
                }
            }
            std::vector<int32_t> next;
            for (int32_t k : cur)
                if (k > js) next.push_back(k);
            if (next.empty()) break;
            if (next.size() == cur.size()) spec = false;
            cur.swap(next);
            CK(upload(h, h->seq, cur, st));
            KL(launch_tail_repass(h->ctl, h->seq.p, (int32_t)cur.size(), n, h->tpiv.p, h->tpinv.p, h->done.p, st));
            CU(cudaMemsetAsync(h->smark.p, 0, (size_t)slots * n * sizeof(int32_t), st));
            if (!bits_smem) CU(cudaMemsetAsync(h->sbits.p, 0, (size_t)slots * words * sizeof(unsigned), st));
            t.seq = h->seq.p;
        }
        if (pool_full) {
            pool *= 2;
            CK(upload(h, h->seq, seq, st));
            continue;
        }
        break;
    }
    if (h->hctl->status != 0) return fail(GBLU_ERR_NOMEM, "restart pool could not be sized");
    h->t_tail[0] = ms_since(t_k);
    const TClock::time_point t_r = TClock::now();
    if (keep_if_same && (int32_t)S.piv.size() == n) {
        // every pivot kept: the structure and schedule stay; only the values
        // of the recomputed columns move from the pool to their slots
        std::vector<int32_t> tp(n);
        CU(cudaMemcpyAsync(tp.data(), h->tpiv.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        if (tp == S.piv) {
            CK(ensure(h, h->sflag, 1));
            CU(cudaMemsetAsync(h->sflag.p, 0, sizeof(int32_t), st));
            KL(launch_pool_scatter(h->seq.p, (int32_t)nR, h->cbeg.p, h->cnu.p, h->cnl.p, h->rows.p, h->LUp.p,
                                   h->LUi.p, h->pinv.p, n, h->vals.p, h->sflag.p, st));
            int32_t bad = 0;
            CU(cudaMemcpyAsync(&bad, h->sflag.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            CU(cudaStreamSynchronize(st));
            if (!bad) {
                h->n_restart_cols = nR;
                h->t_tail[1] = ms_since(t_r);
                h->t_tail[2] = h->t_tail[3] = 0.0;
                return GBLU_OK;
            }
        }
    }
    const unsigned long long top = h->hctl->pool_top;
    // ---- download and repack into the new canonical structure
    std::vector<int32_t> tpiv(n), rows(top);
    std::vector<double> vals(top);
    CU(cudaMemcpyAsync(tpiv.data(), h->tpiv.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(cbeg.data(), h->cbeg.p, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(cnu.data(), h->cnu.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(cnl.data(), h->cnl.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    if (top) {
        CU(cudaMemcpyAsync(rows.data(), h->rows.p, sizeof(int32_t) * top, cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(vals.data(), h->vals.p, sizeof(double) * top, cudaMemcpyDeviceToHost, st));
    }
    CU(cudaStreamSynchronize(st));
    std::vector<int32_t> pinv_new(n, -1);
    for (int32_t k = 0; k < n; k++) {
        if (tpiv[k] < 0 || tpiv[k] >= n || pinv_new[tpiv[k]] >= 0)
            return fail(GBLU_ERR_INTERNAL, "restart produced an invalid pivot sequence");
        pinv_new[tpiv[k]] = k;
    }
    Structure S2;
    S2.n = n;
    S2.piv = tpiv;
    S2.pinv = pinv_new;
    S2.LUp.assign(n + 1, 0);
    S2.nU.assign(n, 0);
    for (int32_t k = 0; k < n; k++) {
        S2.nU[k] = cnu[k];
        S2.LUp[k + 1] = S2.LUp[k] + cnu[k] + cnl[k];
    }
    if (S2.LUp[n] > INT32_MAX) return fail(GBLU_ERR_NOMEM, "factor too large (> 2^31 entries)");
    S2.LUi.resize(S2.LUp[n]);
    std::vector<double> V2(S2.LUp[n]);
    // columns are independent: repack them on several host threads, in
    // ranges of about equal entry counts
    std::atomic<int32_t> misplaced{-1};
    auto repack = [&](int32_t k0, int32_t k1) {
        std::vector<std::pair<int32_t, double>> tmp;
        for (int32_t k = k0; k < k1; k++) {
            const int64_t b = cbeg[k];
            int64_t o = S2.LUp[k];
            // U part: step ids, unchanged numbering for kept columns
            tmp.clear();
            for (int64_t e = b; e < b + cnu[k]; e++)
                tmp.push_back({rmask[k] ? rows[e] : S.LUi[e], vals[e]});
            std::sort(tmp.begin(), tmp.end(), [](auto &x, auto &y) { return x.first < y.first; });
            for (auto &pr : tmp) { S2.LUi[o] = pr.first; V2[o] = pr.second; o++; }
            // L part: original rows (pool) or old step ids (kept) -> new step ids
            tmp.clear();
            for (int64_t e = b + cnu[k]; e < b + cnu[k] + cnl[k]; e++) {
                const int32_t orig = rmask[k] ? rows[e] : S.piv[S.LUi[e]];
                tmp.push_back({pinv_new[orig], vals[e]});
            }
            std::sort(tmp.begin(), tmp.end(), [](auto &x, auto &y) { return x.first < y.first; });
            for (auto &pr : tmp) { S2.LUi[o] = pr.first; V2[o] = pr.second; o++; }
            if (S2.LUi[S2.LUp[k] + S2.nU[k] - 1] != k) misplaced.store(k);
        }
    };
    const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (nt == 1 || n < 4096) {
        repack(0, n);
    } else {
        std::vector<std::thread> pool_threads;
        int32_t k0 = 0;
        for (int t = 1; t <= nt; t++) {
            const int64_t target = S2.LUp[n] * t / nt;
            int32_t k1 = t == nt ? n
                                 : (int32_t)(std::lower_bound(S2.LUp.begin(), S2.LUp.end(), target) - S2.LUp.begin());
            k1 = std::min(std::max(k1, k0), n);
            if (k1 > k0) pool_threads.emplace_back(repack, k0, k1);
            k0 = k1;
        }
        for (auto &th : pool_threads) th.join();
    }
    if (misplaced.load() >= 0)
        return fail(GBLU_ERR_INTERNAL, "restart: diagonal misplaced in column %d", misplaced.load());
    h->n_restart_cols = nR;
    h->t_tail[1] = ms_since(t_r);
    CK(install_structure(h, std::move(S2), &V2, st));
    h->predicted = false;
    return GBLU_OK;
}

// Restart (Section IV-C): every column that did not finish in this
// re-factorization, and all of its column-elimination-tree ancestors, is
// recomputed with pivoting.
// First stage of a restart: the unfinished columns on the installed
// structure, speculating that every step keeps its preferred pivot (the
// previous one), which the threshold check then confirms column by column.
// With every check passing, the structure is the old one (it follows from
// the pattern of A and the pivot order) and the result is exactly the
// factorization with pivoting that prefers the previous pivots; the
// finished columns of the failed pass keep their values.  A column whose
// check fails again needs another pivot: *interrupted = 1, and the columns
// finished by now stay final for the pivoting stage.
// With no_stop, a failing column does not end the launch: every column is
// computed, so first_bad is the first step whose check fails (every column
// before it passed), and that column holds its unnormalized values for the
// pivot choice of a re-prediction.
int restart_on_structure(gblu_ctx *h, const double *Ax, cudaStream_t st, bool no_stop, int *interrupted)
{
    KL(launch_begin_refactor(h->ctl, st));
    RefactorArgs a = refactor_args(h, Ax);
    a.force_col = -1;
    a.skip_done = 1;
    a.no_stop = no_stop ? 1 : 0;
    a.task_begin = 0;
    a.ntasks = (int32_t)h->W.task_ptr.size() - 1;
    KL(launch_refactor_tasks(a, true, pgrid(h, h->ref_blocks_per_sm), h->epoch, st));
    CK(read_ctl(h, st));
    CK(status_code(h));
    *interrupted = h->hctl->interrupted || h->hctl->first_bad != INT_MAX;
    return GBLU_OK;
}

// Restart by re-prediction (Section IV-C/D, with the threshold rule of
// Section II-A).  On entry the installed structure is a symmetric prediction
// for the pivot rows it holds (pred), every step before k passed its check,
// and column k, whose check failed, holds its unnormalized values.  The
// threshold rule then takes at step k the candidate of largest magnitude,
// the row of some later step s; s is predicted to take k's row in exchange
// (the row that a kept step s would otherwise lose is k's), the structure is
// predicted again for the new rows (the Cholesky pattern of B + B^T, B =
// A(pred, Q)), and the checked re-factorization computes every column in
// no-stop mode.  Where a step's predicted row is not its preferred one
// (prefer), the rule takes the largest candidate, so its check asks for a
// strict maximum (strict_col).  Steps before the first failure keep their
// rows and values, so every round moves the first failure forward.  *solved
// = false after kMaxRepredict rounds, a non-finite or all-zero candidate
// set, a round without progress or a structure that grows past a quarter of
// the preferred one: the caller then runs the pivoting kernel.
constexpr int kMaxRepredict = 6;

int repredict(gblu_ctx *h, const double *Ax, cudaStream_t st, const std::vector<int32_t> &prefer, int32_t k,
              bool *solved)
{
    *solved = false;
    h->repredictions = 0;
    // a forced failure (gblu_refactorize_forced) belongs to the first pass
    // only; the rounds check every column as it is
    struct ForceOff {
        gblu_ctx *h;
        int32_t saved;
        ~ForceOff() { h->force_col = saved; }
    } force_off{h, h->force_col};
    h->force_col = -1;
    const int32_t n = h->P.n;
    const int64_t nnz_limit = h->S.nnz() + h->S.nnz() / 4 + n;
    // the failing step reported for the call is the first check's
    const int32_t first_bad = h->last_first_bad;
    std::vector<int32_t> pred = h->S.piv;
    std::vector<uint8_t> strict(n, 0);
    for (int32_t j = 0; j < n; j++) strict[j] = pred[j] != prefer[j];
    CK(ensure(h, h->pchoice, 2));
    for (int round = 0; round < kMaxRepredict; round++) {
        if (k < 0 || k >= n) return GBLU_OK;
        KL(launch_pivot_choice(h->LUp.p, h->LUi.p, h->vals.p, h->nU.p, h->piv.p, h->qinv.p, k, h->pchoice.p, st));
        int32_t ch[2] = {-1, 0};
        CU(cudaMemcpyAsync(ch, h->pchoice.p, sizeof ch, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        const int32_t s = ch[0];
        if (ch[1] || s <= k || s >= n) return GBLU_OK;
        std::swap(pred[k], pred[s]);
        strict[k] = pred[k] != prefer[k];
        strict[s] = pred[s] != prefer[s];
        Structure S2;
        symmetric_structure(h->P, S2, &pred);
        if (S2.nnz() > nnz_limit) return GBLU_OK;
        CK(install_structure(h, std::move(S2), nullptr, st, true));
        h->predicted = true;
        CK(upload(h, h->strict, strict, st));
        h->strict_on = true;
        h->no_stop = true;
        int interrupted = 0;
        const int rc = run_refactor(h, Ax, st, &interrupted);
        h->strict_on = false;
        h->no_stop = false;
        h->last_first_bad = first_bad;
        CK(rc);
        h->repredictions = round + 1;
        const int32_t kn = h->hctl->first_bad;
        if (kn == INT_MAX) {
            *solved = true;
            return GBLU_OK;
        }
        if (kn <= k) return GBLU_OK;
        k = kn;
    }
    return GBLU_OK;
}

// Every step recomputed by the pivoting kernel, preferring the rows
// prefer[k] (the definition of a factorization with preferred pivots, used
// when a re-prediction gives up)
int pivot_every_step(gblu_ctx *h, const double *Ax, cudaStream_t st, const std::vector<int32_t> &prefer)
{
    const int32_t n = h->P.n;
    Structure E;
    E.n = n;
    E.LUp.assign(n + 1, 0);
    E.nU.assign(n, 0);
    E.piv = prefer;
    E.pinv.assign(n, -1);
    for (int32_t k = 0; k < n; k++) E.pinv[prefer[k]] = k;
    h->S = std::move(E);
    CK(upload(h, h->piv, h->S.piv, st));
    CK(upload(h, h->pinv, h->S.pinv, st));
    const size_t hint = (size_t)(1.25 * (double)(2 * symmetric_fill(h->P) + n));
    std::vector<uint8_t> all(n, 1);
    return run_tail(h, Ax, st, all, hint, false, true);
}

// The pivot moves of a restart on a predicted structure, from the first
// failing step k of a no-stop pass (Section IV-C/D): re-prediction, else
// the pivoting kernel over every step, with the installed pivots preferred.
int restart_repredicted(gblu_ctx *h, const double *Ax, cudaStream_t st, int32_t k,
                        std::chrono::steady_clock::time_point t0)
{
    const std::vector<int32_t> prefer = h->S.piv;
    bool solved = false;
    CK(repredict(h, Ax, st, prefer, k, &solved));
    if (!solved) CK(pivot_every_step(h, Ax, st, prefer));
    h->n_restart_cols = h->P.n;
    if (solved) h->tail_passes = 0;
    h->t_tail[0] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (solved) h->t_tail[1] = h->t_tail[3] = 0.0;
    return GBLU_OK;
}

int run_restart(gblu_ctx *h, const double *Ax, cudaStream_t st)
{
    NvtxRange nvtx_range("restart");
    const int32_t n = h->P.n;
    h->repredictions = 0;
    if (h->W.dense_m == 0) {
        const auto t0 = std::chrono::steady_clock::now();
        std::vector<int32_t> fin0(n);
        CU(cudaMemcpyAsync(fin0.data(), h->finish.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        int interrupted = 0;
        // on a predicted structure a pivot that must move is found exactly
        // (no-stop) and re-predicted; on another structure the restart set
        // goes to the pivoting kernel
        const bool repred = h->predicted;
        CK(restart_on_structure(h, Ax, st, repred, &interrupted));
        if (interrupted && repred) return restart_repredicted(h, Ax, st, h->hctl->first_bad, t0);
        if (!interrupted) {
            int64_t redone = 0;
            for (int32_t k = 0; k < n; k++) redone += fin0[k] != h->epoch;
            h->n_restart_cols = redone;
            h->tail_passes = 0;
            h->t_tail[0] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            h->t_tail[1] = h->t_tail[2] = h->t_tail[3] = 0.0;
            return GBLU_OK;
        }
    }
    std::vector<int32_t> fin(n);
    CU(cudaMemcpyAsync(fin.data(), h->finish.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    std::vector<uint8_t> finished(n), rmask(n);
    for (int32_t k = 0; k < n; k++) finished[k] = fin[k] == h->epoch;
    gblu_restart_set(n, h->P.cetree.data(), finished.data(), rmask.data());
    return run_tail(h, Ax, st, rmask, 0, true, true);
}

int check_handle(gblu_ctx *h)
{
    if (!h) return fail(GBLU_ERR_INVALID_INPUT, "null handle");
    if (!h->analyzed) return fail(GBLU_ERR_NOT_ANALYZED, "gblu_analyze has not been called");
    return GBLU_OK;
}

}  // namespace

// =========================================================================== C ABI
extern "C" {

void gblu_default_opts(gblu_opts *o)
{
    if (!o) return;
    o->pivot_tol = 1e-3;
    o->sched_mode = GBLU_SCHED_AUTO;
    o->solve_mode = GBLU_SCHED_AUTO;
    o->alpha = 2.0;
    o->spin_limit = 1LL << 24;
    o->solve_dense_frac = 0.7;
    o->solve_dense_min = 300000;
    o->solve_slices = 8;
    o->solve_dense_density = 0.9;
    o->dense_min_rows = 0;
    o->warp_column_max = kRefCapShort;
    o->speculate_first = 2;
    o->batch_group = 0;
    o->solve_ctas_per_sm = 0;
    o->max_sms = 0;
}

const char *gblu_last_error(void) { return g_err.c_str(); }

static bool opts_valid(const gblu_opts &o)
{
    return o.pivot_tol >= 0.0 && o.pivot_tol <= 1.0 && o.spin_limit > 0 && o.sched_mode >= 0 && o.sched_mode <= 2 &&
           o.solve_mode >= 0 && o.solve_mode <= 2 && o.alpha >= 0.0 && o.solve_dense_frac >= 0.0 &&
           o.solve_dense_frac <= 1.0 && o.solve_slices >= 0 && o.solve_dense_density >= 0.0 &&
           o.solve_dense_density <= 1.0 && o.dense_min_rows >= 0 && o.warp_column_max >= 32 &&
           o.warp_column_max <= kRefCapShort && (o.speculate_first >= 0 && o.speculate_first <= 2) &&
           o.batch_group >= 0 && o.solve_ctas_per_sm >= 0 && o.max_sms >= 0;
}

int gblu_create(gblu_handle *out, int device, const gblu_opts *o)
{
    if (!out) return fail(GBLU_ERR_INVALID_INPUT, "null output pointer");
    *out = nullptr;
    gblu_ctx *h = new (std::nothrow) gblu_ctx();
    if (!h) return fail(GBLU_ERR_NOMEM, "host allocation failed");
    gblu_default_opts(&h->opts);
    if (o) h->opts = *o;
    if (!opts_valid(h->opts)) {
        delete h;
        return fail(GBLU_ERR_INVALID_INPUT, "invalid options");
    }
    h->device = device;
    DeviceGuard g(device);
    if (!g.ok) {
        delete h;
        return fail(GBLU_ERR_CUDA, "cannot use CUDA device %d", device);
    }
    cudaError_t e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->l2_bytes, cudaDevAttrL2CacheSize, device);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hctl, sizeof(DevCtl));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->ctl, sizeof(DevCtl));
    if (e == cudaSuccess) e = cudaMemset(h->ctl, 0, sizeof(DevCtl));
    int r = 0;
    if (e == cudaSuccess) r = refactor_setup(kRefCapLong, &h->ref_blocks_per_sm, &h->batch_blocks_per_sm);
    if (e == cudaSuccess && r == 0) r = refactor_setup_f32(kRefCapLong, &h->ref32_blocks_per_sm);
    if (e == cudaSuccess && r == 0) r = solve_syncfree_grid(&h->solve_grid);
    int trail_per_sm = 0;
    if (e == cudaSuccess && r == 0) r = trail_setup(&trail_per_sm);
    if (e == cudaSuccess && r == 0) r = dense_setup(GBLU_DENSE_MAX_ROWS);
    if (e == cudaSuccess && r == 0) r = tail_setup();
    if (e != cudaSuccess || r != 0 || h->ref_blocks_per_sm < 1 || h->batch_blocks_per_sm < 1) {
        const char *msg = cudaGetErrorString(e != cudaSuccess ? e : (cudaError_t)r);
        if (h->hctl) cudaFreeHost(h->hctl);
        if (h->ctl) cudaFree(h->ctl);
        delete h;
        cudaGetLastError();
        return fail(GBLU_ERR_CUDA, "device setup failed: %s", msg);
    }
    h->ref_grid = h->ref_blocks_per_sm * h->sm_count;
    h->ref32_grid = h->ref32_blocks_per_sm * h->sm_count;
    h->res_blocks = h->sm_count * 4;
    h->trail_per_sm = std::max(1, trail_per_sm);
    *out = h;
    return GBLU_OK;
}

void gblu_destroy(gblu_handle h)
{
    if (!h) return;
    {
        DeviceGuard g(h->device);
        cudaDeviceSynchronize();
        release(h, h->Ap); release(h, h->Ai); release(h, h->Q); release(h, h->qinv);
        release(h, h->clo); release(h, h->Acol); release(h, h->Aslot); release(h, h->Arp);
        release(h, h->LUp); release(h, h->LUi); release(h, h->nU); release(h, h->rows); release(h, h->chain);
        release(h, h->finish); release(h, h->task_ptr); release(h, h->task_cols); release(h, h->amap);
        release(h, h->piv); release(h, h->pinv); release(h, h->vals);
        release(h, h->Lrp); release(h, h->Urp); release(h, h->Lcol); release(h, h->Lslot);
        release(h, h->Ucol); release(h, h->Uslot); release(h, h->Udiag);
        release(h, h->lsv_rows); release(h, h->usv_rows); release(h, h->lbs); release(h, h->ubs);
        release(h, h->lrb); release(h, h->urb); release(h, h->lsv_tick); release(h, h->usv_tick);
        release(h, h->ext_l); release(h, h->ext_u); release(h, h->dense); release(h, h->dense_s0);
        release(h, h->bfinish); release(h, h->bticket); release(h, h->bctl); release(h, h->bargs);
        release(h, h->vals32); release(h, h->vals_w); release(h, h->ir_r); release(h, h->ir_d); release(h, h->ir_out);
        if (h->ir_host) cudaFreeHost(h->ir_host);
        release(h, h->lseg);
        release(h, h->useg); release(h, h->ltri0); release(h, h->ufar); release(h, h->far);
        release(h, h->y); release(h, h->z); release(h, h->partial);
        release(h, h->stage_ax); release(h, h->stage_b); release(h, h->stage_x);
        release(h, h->seq); release(h, h->restart); release(h, h->done); release(h, h->tpiv);
        release(h, h->tpinv); release(h, h->cnu); release(h, h->cnl); release(h, h->smark);
        release(h, h->slist); release(h, h->sclass); release(h, h->cbeg); release(h, h->sx);
        release(h, h->sflag); release(h, h->sbits); release(h, h->morder); release(h, h->mlorder);
        release(h, h->muorder); release(h, h->margs); release(h, h->mticket);
        if (h->gexec) cudaGraphExecDestroy(h->gexec);
        if (h->bgexec) cudaGraphExecDestroy(h->bgexec);
        if (h->bgctl_host) cudaFreeHost(h->bgctl_host);
        release(h, h->bgargs);
        if (h->gstream) cudaStreamDestroy(h->gstream);
        if (h->aux) cudaStreamDestroy(h->aux);
        if (h->epoch_host) cudaFreeHost(h->epoch_host);
        if (h->ctl) cudaFree(h->ctl);
        if (h->hctl) cudaFreeHost(h->hctl);
    }
    delete h;
}

int gblu_analyze(gblu_handle h, int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *Q)
{
    if (!h) return fail(GBLU_ERR_INVALID_INPUT, "null handle");
    std::string err;
    int rc = validate_pattern(n, Ap, Ai, err);
    if (rc != GBLU_OK) return fail(rc, "invalid pattern: %s", err.c_str());
    DeviceGuard g(h->device);
    if (!g.ok) return fail(GBLU_ERR_CUDA, "cannot use CUDA device %d", h->device);
    h->analyzed = false;
    h->factorized = false;
    Pattern &P = h->P;
    P = Pattern();
    P.n = n;
    P.Ap.assign(Ap, Ap + n + 1);
    P.Ai.assign(Ai, Ai + Ap[n]);
    P.Q.assign(n, 0);
    if (Q) {
        std::vector<uint8_t> seen(n, 0);
        for (int32_t k = 0; k < n; k++) {
            if (Q[k] < 0 || Q[k] >= n || seen[Q[k]]) return fail(GBLU_ERR_INVALID_INPUT, "Q is not a permutation");
            seen[Q[k]] = 1;
            P.Q[k] = Q[k];
        }
    } else {
        auto_order(n, Ap, Ai, P.Q.data());
    }
    P.qinv.assign(n, 0);
    for (int32_t k = 0; k < n; k++) P.qinv[P.Q[k]] = k;
    column_etree(P, P.cetree);
    P.clo.resize(n);
    std::vector<int32_t> depth(n, 0);
    for (int32_t k = 0; k < n; k++) P.clo[k] = k;
    for (int32_t k = 0; k < n; k++) {
        const int32_t p = P.cetree[k];
        if (p >= 0) P.clo[p] = std::min(P.clo[p], P.clo[k]);
    }
    P.cetree_height = 0;
    for (int32_t k = n - 1; k >= 0; k--) {
        const int32_t p = P.cetree[k];
        depth[k] = p >= 0 ? depth[p] + 1 : 1;
        P.cetree_height = std::max(P.cetree_height, depth[k]);
    }
    // row-wise copy of A for the residual
    P.Arp.assign(n + 1, 0);
    for (int32_t p = 0; p < Ap[n]; p++) P.Arp[Ai[p] + 1]++;
    for (int32_t i = 0; i < n; i++) P.Arp[i + 1] += P.Arp[i];
    P.Acol.assign(Ap[n], 0);
    P.Aslot.assign(Ap[n], 0);
    {
        std::vector<int64_t> pos(P.Arp.begin(), P.Arp.end() - 1);
        for (int32_t c = 0; c < n; c++)
            for (int32_t p = Ap[c]; p < Ap[c + 1]; p++) {
                P.Acol[pos[Ai[p]]] = c;
                P.Aslot[pos[Ai[p]]++] = p;
            }
    }
    cudaStream_t st = 0;
    CK(upload(h, h->Ap, P.Ap, st));
    CK(upload(h, h->Ai, P.Ai, st));
    CK(upload(h, h->Q, P.Q, st));
    CK(upload(h, h->qinv, P.qinv, st));
    CK(upload(h, h->clo, P.clo, st));
    CK(upload(h, h->Arp, P.Arp, st));
    CK(upload(h, h->Acol, P.Acol, st));
    CK(upload(h, h->Aslot, P.Aslot, st));
    CK(ensure(h, h->partial, (size_t)3 * h->res_blocks));
    CU(cudaStreamSynchronize(st));
    h->analyzed = true;
    return GBLU_OK;
}

// The predicted structure is a superset of the exact one by the fill that
// the unsymmetric entries of A add; with at most 2% of the off-diagonal
// entries unsymmetric it stays close (0.1% more entries on the RC meshes
// with transistors, whose transconductance entries are the unsymmetric ones)
static bool nearly_symmetric(const Pattern &P)
{
    const int64_t offdiag = (int64_t)P.Ai.size() - P.n;
    return offdiag <= 0 || unsymmetric_entries(P) * 50 <= offdiag;
}

int gblu_factorize(gblu_handle h, const double *Ax_dev, void *stream)
{
    NvtxRange nvtx_range("gblu_factorize");
    CK(check_handle(h));
    h->last_repivot = false;
    if (!Ax_dev) return fail(GBLU_ERR_INVALID_INPUT, "null Ax_dev");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    h->factorized = false;
    // no kept columns: an empty structure whose preferred pivots are the
    // diagonal rows Q[k]; every step is computed with pivoting, in passes
    // that speculate that each step takes its diagonal row
    const int32_t n = h->P.n;
    Structure S;
    S.n = n;
    S.LUp.assign(n + 1, 0);
    S.nU.assign(n, 0);
    S.LUi.clear();
    S.piv = h->P.Q;
    S.pinv = h->P.qinv;
    h->S = std::move(S);
    CK(upload(h, h->piv, h->S.piv, st));
    CK(upload(h, h->pinv, h->S.pinv, st));
    bool spec = h->opts.speculate_first != 0;
    int64_t zero_diag = 0;
    if (spec && n > 0) {
        // the prediction fails where A's diagonal entry is absent or zero
        // (the branch rows of MNA voltage sources) unless fill makes it
        // nonzero: with more such steps than a pass tolerates, every step
        // waits in order from the start
        const std::vector<int32_t> &Ap = h->P.Ap, &Ai = h->P.Ai;
        std::vector<double> ax(Ai.size());
        if (!ax.empty())
            CU(cudaMemcpyAsync(ax.data(), Ax_dev, sizeof(double) * ax.size(), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        for (int32_t k = 0; k < n && zero_diag <= kSpecMaxMoved; k++) {
            const int32_t c = h->P.Q[k];
            bool nz = false;
            for (int32_t p = Ap[c]; p < Ap[c + 1] && !nz; p++) nz = Ai[p] == c && ax[p] != 0.0;
            zero_diag += !nz;
        }
        spec = zero_diag <= kSpecMaxMoved;
    }
    CU(cudaStreamSynchronize(st));
    h->first_mode = 0;
    h->t_first_symbolic = 0.0;
    h->predicted = false;
    h->repredictions = 0;
    if (spec && h->opts.speculate_first == 2 && zero_diag == 0 && nearly_symmetric(h->P)) {
        // the prediction as a structure: L and U^T with the pattern of the
        // Cholesky factor of (A + A^T)(Q,Q), which holds the pattern of the
        // factors when every step keeps its diagonal row; the checked
        // re-factorization kernel then computes every column, and the check
        // is the threshold rule with the diagonal preferred (Algorithm 1)
        const auto t0 = std::chrono::steady_clock::now();
        Structure S2;
        symmetric_structure(h->P, S2);
        h->t_first_symbolic = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        CK(install_structure(h, std::move(S2), nullptr, st, true));
        h->predicted = true;
        const auto t1 = std::chrono::steady_clock::now();
        int interrupted = 0;
        h->force_col = -1;
        // no-stop: a failing step does not end the launch, so the first one
        // is known exactly and its column keeps its values for the pivot
        // choice (the dense tail's block checks its columns itself, so with
        // a dense tail a failure stops the launch as in a re-factorization)
        const bool repred = h->W.dense_m == 0;
        h->no_stop = repred;
        const int rc = run_refactor(h, Ax_dev, st, &interrupted);
        h->no_stop = false;
        CK(rc);
        h->t_tail[0] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
        h->t_tail[1] = 0.0;
        h->tail_passes = 0;
        h->n_restart_cols = 0;
        h->first_mode = 1;
        if (!repred && interrupted) {
            // the unfinished steps and their column-elimination-tree
            // ancestors go through the pivoting kernel, as in the second
            // stage of a restart (Section IV-C); the finished steps kept
            // their diagonal rows
            std::vector<int32_t> fin(n);
            CU(cudaMemcpyAsync(fin.data(), h->finish.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
            CU(cudaStreamSynchronize(st));
            std::vector<uint8_t> finished(n), rmask(n);
            for (int32_t k = 0; k < n; k++) finished[k] = fin[k] == h->epoch;
            gblu_restart_set(n, h->P.cetree.data(), finished.data(), rmask.data());
            CK(run_tail(h, Ax_dev, st, rmask, 0, true, true));
            h->first_mode = 2;
        } else if (repred && h->hctl->first_bad != INT_MAX) {
            h->last_first_bad = h->hctl->first_bad;
            // a step needs another row: the structure is predicted again for
            // the rows the threshold rule takes (the restart's re-prediction,
            // with the diagonal rows preferred); if that gives up, the
            // pivoting kernel computes every step
            bool solved = false;
            CK(repredict(h, Ax_dev, st, h->P.Q, h->hctl->first_bad, &solved));
            if (solved) {
                h->first_mode = 3;
            } else {
                CK(pivot_every_step(h, Ax_dev, st, h->P.Q));
                h->first_mode = 2;
            }
        }
        h->factorized = true;
        return GBLU_OK;
    }
    const size_t hint = (size_t)(1.25 * (double)(2 * symmetric_fill(h->P) + n));
    std::vector<uint8_t> all(n, 1);
    CK(run_tail(h, Ax_dev, st, all, hint, false, spec));
    h->factorized = true;
    return GBLU_OK;
}

int gblu_last_status(gblu_handle h, void *stream)
{
    CK(check_handle(h));
    DeviceGuard g(h->device);
    CK(read_ctl(h, (cudaStream_t)stream));
    if (h->hctl->status != 0) return status_code(h);
    return h->last_repivot ? GBLU_REPIVOTED : GBLU_OK;
}

int gblu_refactorize_forced(gblu_handle h, const double *Ax_dev, void *stream, int32_t force_col,
                            int32_t *repivoted)
{
    CK(check_handle(h));
    if (repivoted) *repivoted = 0;
    if (force_col < -1 || force_col >= h->P.n)
        return fail(GBLU_ERR_INVALID_INPUT, "force_col %d outside [-1, n)", force_col);
    h->force_col = force_col;
    const int rc = gblu_refactorize(h, Ax_dev, stream, repivoted);
    h->force_col = -1;
    return rc;
}

int gblu_refactorize(gblu_handle h, const double *Ax_dev, void *stream, int32_t *repivoted)
{
    NvtxRange nvtx_range("gblu_refactorize");
    CK(check_handle(h));
    h->last_repivot = false;
    if (repivoted) *repivoted = 0;
    if (!h->factorized) return fail(GBLU_ERR_NOT_FACTORIZED, "gblu_factorize has not succeeded");
    if (!Ax_dev) return fail(GBLU_ERR_INVALID_INPUT, "null Ax_dev");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    int interrupted = 0;
    h->n_refactor++;
    // On a predicted structure a failed check needs a pivot to move: the
    // restart's first stage would meet the same failure (the same values,
    // dependencies and order), unless the failure was forced.  The pass
    // then runs in no-stop mode, so the first failing step is exact and its
    // column holds the values for the pivot choice, and the restart goes
    // straight to re-prediction.
    const bool direct = h->predicted && h->force_col < 0 && h->W.dense_m == 0;
    const auto t0 = std::chrono::steady_clock::now();
    h->no_stop = direct;
    int rc = run_refactor(h, Ax_dev, st, &interrupted);
    h->no_stop = false;
    if (rc != GBLU_OK) {
        h->factorized = false;
        return rc;
    }
    if (direct && h->hctl->first_bad != INT_MAX) {
        NvtxRange nvtx_range("restart");
        h->n_repivot++;
        h->repredictions = 0;
        h->last_first_bad = h->hctl->first_bad;
        rc = restart_repredicted(h, Ax_dev, st, h->hctl->first_bad, t0);
        if (rc != GBLU_OK) {
            h->factorized = false;
            return rc;
        }
        if (repivoted) *repivoted = 1;
        h->last_repivot = true;
        return GBLU_REPIVOTED;
    }
    if (!interrupted) return GBLU_OK;
    h->n_repivot++;
    rc = run_restart(h, Ax_dev, st);
    if (rc != GBLU_OK) {
        h->factorized = false;
        return rc;
    }
    if (repivoted) *repivoted = 1;
    h->last_repivot = true;
    return GBLU_REPIVOTED;
}

// both triangular solves of nsets systems on the installed structure: set s
// with factor values LUx + s*lu_stride, right-hand side b_dev + s*b_stride,
// solution x_dev + s*x_stride
// solve arguments of one system on the handle's structure (the row-block
// fields are set per triangle by the caller)
static SolveArgs solve_args(gblu_ctx *h, const double *LUx, const double *b_dev, double *x_dev)
{
    SolveArgs a{};
    a.n = h->S.n;
    a.LUx = LUx;
    a.nsets = 1;
    a.v_stride = h->S.n;
    a.Lrp = h->Lrp.p;
    a.Urp = h->Urp.p;
    a.Lcol = h->Lcol.p;
    a.Lslot = h->Lslot.p;
    a.Ucol = h->Ucol.p;
    a.Uslot = h->Uslot.p;
    a.Udiag = h->Udiag.p;
    a.piv = h->piv.p;
    a.Q = h->Q.p;
    a.b = b_dev;
    a.y = h->y.p;
    a.z = h->z.p;
    a.x = x_dev;
    a.spin_limit = h->opts.spin_limit;
    a.ctl = h->ctl;
    return a;
}

// grid of the sync-free solve launches: the option's CTAs per SM, at most
// as many as fit
static int solve_grid(gblu_ctx *h)
{
    const int fit = h->solve_grid / std::max(1, h->sm_count);   // CTAs per SM that fit
    const int per = h->opts.solve_ctas_per_sm;
    return pgrid(h, (per <= 0 || per >= fit) ? fit : per);
}

static int solve_values(gblu_ctx *h, const double *LUx, int64_t lu_stride, const double *b_dev, int64_t b_stride,
                        double *x_dev, int64_t x_stride, int32_t nsets, cudaStream_t st)
{
    const int32_t n = h->S.n;
    if (nsets > 1) {   // per-set intermediate vectors
        if ((int64_t)n * nsets > INT_MAX) return fail(GBLU_ERR_INVALID_INPUT, "batch too large");
        CK(ensure(h, h->y, (size_t)n * nsets));
        CK(ensure(h, h->z, (size_t)n * nsets));
        CK(ensure(h, h->ext_l, (size_t)n * nsets));
        CK(ensure(h, h->ext_u, (size_t)n * nsets));
        if (h->W.up0 < n) CK(ensure(h, h->far, (size_t)n * nsets));
    }
    KL(launch_begin_solve(h->ctl, h->y.p, h->z.p, h->ext_l.p, h->ext_u.p, n * nsets, st));
    SolveArgs a = solve_args(h, LUx, b_dev, x_dev);
    a.nsets = nsets;
    a.lu_stride = lu_stride;
    a.b_stride = b_stride;
    a.x_stride = x_stride;
    const Schedule &W = h->W;
    // sparse part (rows [0, lp0) / [0, up0)) in row blocks: block levels
    // before the dividing level one launch each, the rest one sync-free launch
    auto sparse = [&](bool lower) -> int {
        const std::vector<int32_t> &ptr = lower ? W.lsv_ptr : W.usv_ptr;     // blocks per level
        const std::vector<int32_t> &tptr = lower ? W.lsv_tptr : W.usv_tptr;  // rows per level
        const int32_t nlev = lower ? W.lsv_levels : W.usv_levels;
        const int32_t nrows = (int32_t)(lower ? W.lsv_tick.size() : W.usv_tick.size());
        int32_t div = lower ? W.lsv_div : W.usv_div;
        if (h->opts.solve_mode == GBLU_SCHED_LEVEL) div = nlev;
        if (h->opts.solve_mode == GBLU_SCHED_SYNCFREE) div = 0;
        int32_t *blocks = lower ? h->lsv_rows.p : h->usv_rows.p;
        int32_t *tick = lower ? h->lsv_tick.p : h->usv_tick.p;
        a.bs = lower ? h->lbs.p : h->ubs.p;
        a.rb = lower ? h->lrb.p : h->urb.p;
        a.ext = lower ? h->ext_l.p : h->ext_u.p;
        for (int32_t l = 0; l < div; l++) {   // outside sums of the level's rows, then its blocks
            a.rows = tick + tptr[l];
            a.nrows = tptr[l + 1] - tptr[l];
            KL(lower ? launch_lsolve(a, true, 0, st) : launch_usolve(a, true, 0, st));
            a.rows = blocks + ptr[l];
            a.nrows = ptr[l + 1] - ptr[l];
            KL(launch_solve_finish(a, lower, st));
        }
        if (div < nlev) {
            a.rows = tick + tptr[div];
            a.nrows = nrows - tptr[div];
            KL(lower ? launch_lsolve(a, false, solve_grid(h), st)
                     : launch_usolve(a, false, solve_grid(h), st));
        }
        return GBLU_OK;
    };
    // forward: sparse row blocks, then the trailing block (its rows' sums
    // over earlier columns, then its 32-row slices sync-free)
    CK(sparse(true));
    if (W.lp0 < n) {
        const TrailArgs t{W.lp0, n, W.lnb, h->lseg.p, h->LUp.p, h->LUi.p, h->nU.p, h->ltri0.p};
        a.ext = h->ext_l.p;
        KL(launch_trail(a, t, true, pgrid(h, h->trail_per_sm), st));
        h->launches++;   // two kernels
    }
    // backward: the trailing block's slices, then the sums of the rows above
    // it over its columns, then the sparse row blocks
    if (W.up0 < n) {
        const TrailArgs t{W.up0, n, W.unb, h->useg.p, h->LUp.p, h->LUi.p, h->nU.p, h->ufar.p};
        a.far = h->far.p;
        KL(launch_trail(a, t, false, pgrid(h, h->trail_per_sm), st));
        if (W.up0 > 0) h->launches++;
        a.ufar = h->ufar.p;
    }
    CK(sparse(false));
    return GBLU_OK;
}

int gblu_solve(gblu_handle h, const double *b_dev, double *x_dev, void *stream)
{
    NvtxRange nvtx_range("gblu_solve");
    CK(check_handle(h));
    if (!h->factorized) return fail(GBLU_ERR_NOT_FACTORIZED, "no valid factorization");
    if (!b_dev || !x_dev) return fail(GBLU_ERR_INVALID_INPUT, "null vector");
    DeviceGuard g(h->device);
    return solve_values(h, h->vals.p, 0, b_dev, 0, x_dev, 0, 1, (cudaStream_t)stream);
}

// sets per group of a batch's persistent launch: the option, else as many
// sets as fit in half of L2 (their factor and A values)
static int batch_group(gblu_ctx *h, int32_t nsets)
{
    int g = h->opts.batch_group;
    if (g <= 0) {
        const double per = 8.0 * ((double)h->S.nnz() + (double)h->P.Ai.size());
        g = (int)std::max(1.0, 0.5 * (double)h->l2_bytes / std::max(per, 1.0));
    }
    return std::min(g, (int)nsets);
}

int gblu_refactorize_batch(gblu_handle h, int32_t nsets, const double *Ax_dev, int64_t ax_stride,
                           double *LUx_dev, int64_t lu_stride, int32_t *failed, int32_t *n_failed,
                           void *stream)
{
    NvtxRange nvtx_range("gblu_refactorize_batch");
    CK(check_handle(h));
    if (n_failed) *n_failed = 0;
    if (!h->factorized) return fail(GBLU_ERR_NOT_FACTORIZED, "gblu_factorize has not succeeded");
    const int64_t nnz_a = (int64_t)h->P.Ai.size(), nnz = h->S.nnz();
    if (nsets < 1 || !Ax_dev || !LUx_dev || ax_stride < nnz_a || lu_stride < nnz)
        return fail(GBLU_ERR_INVALID_INPUT, "batch: nsets >= 1, non-null buffers, strides >= %lld and %lld",
                    (long long)nnz_a, (long long)nnz);
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t n = h->S.n;
    const size_t fcap = h->bfinish.cap;
    CK(ensure(h, h->bfinish, (size_t)nsets * n));
    if (h->bfinish.cap != fcap)   // fresh flags: epochs start above zero
        CU(cudaMemsetAsync(h->bfinish.p, 0, h->bfinish.cap * sizeof(int32_t), st));
    CK(ensure(h, h->bctl, (size_t)nsets));
    CK(ensure(h, h->bargs, (size_t)nsets));
    CK(ensure(h, h->bticket, 1));
    h->epoch++;
    h->n_refactor += nsets;
    const RefactorArgs base = refactor_args(h, nullptr);
    h->bargs_host.assign(nsets, base);
    for (int32_t s = 0; s < nsets; s++) {
        RefactorArgs &as = h->bargs_host[s];
        as.Ax = Ax_dev + s * ax_stride;
        as.LUx = LUx_dev + s * lu_stride;
        as.finish = h->bfinish.p + (size_t)s * n;
        as.ctl = h->bctl.p + s;
        as.dense_p = INT_MAX;   // the dense tail is not used in batches
    }
    CU(cudaMemcpyAsync(h->bargs.p, h->bargs_host.data(), sizeof(RefactorArgs) * nsets, cudaMemcpyHostToDevice, st));
    KL(launch_begin_batch(h->bctl.p, nsets, h->bticket.p, st));
    RefactorArgs a0 = base;
    const std::vector<int32_t> &ltp = h->W.level_task_ptr;
    const int32_t div = h->W.div_level;
    for (int32_t l = 0; l < div; l++) {   // cluster mode
        a0.task_begin = ltp[l];
        a0.ntasks = ltp[l + 1] - ltp[l];
        KL(launch_refactor_batch(h->bargs.p, a0, nsets, false, 0, h->epoch, h->bticket.p, st, nsets));
    }
    const int32_t ntask = (int32_t)h->W.task_ptr.size() - 1;
    if (ltp[div] < ntask) {               // pipeline mode
        a0.task_begin = ltp[div];
        a0.ntasks = ntask - ltp[div];
        KL(launch_refactor_batch(h->bargs.p, a0, nsets, true, pgrid(h, h->batch_blocks_per_sm), h->epoch, h->bticket.p, st,
                                 batch_group(h, nsets)));
    }
    h->bctl_host.resize(nsets);
    CU(cudaMemcpyAsync(h->bctl_host.data(), h->bctl.p, sizeof(DevCtl) * nsets, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    int32_t nf = 0;
    for (int32_t s = 0; s < nsets; s++) {
        const DevCtl &c = h->bctl_host[s];
        if (c.status != 0) return fail(c.status, "batch set %d: device status %d (wait %d at column %d)", s,
                                       c.status, c.where, c.where_k);
        if (failed) failed[s] = c.interrupted ? 1 : 0;
        nf += c.interrupted ? 1 : 0;
    }
    if (n_failed) *n_failed = nf;
    return GBLU_OK;
}

int gblu_solve_batch(gblu_handle h, int32_t nsets, const double *LUx_dev, int64_t lu_stride,
                     const double *b_dev, int64_t b_stride, double *x_dev, int64_t x_stride, void *stream)
{
    NvtxRange nvtx_range("gblu_solve_batch");
    CK(check_handle(h));
    if (!h->factorized) return fail(GBLU_ERR_NOT_FACTORIZED, "no valid factorization");
    const int32_t n = h->S.n;
    if (nsets < 1 || !LUx_dev || !b_dev || !x_dev || lu_stride < h->S.nnz() || b_stride < n || x_stride < n)
        return fail(GBLU_ERR_INVALID_INPUT, "batch solve: nsets >= 1, non-null buffers, strides too small");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    return solve_values(h, LUx_dev, lu_stride, b_dev, b_stride, x_dev, x_stride, nsets, st);
}

int gblu_refactorize_multi(int32_t nh, gblu_handle *hs, const double *const *Ax_dev, void *stream,
                           int32_t *repivoted)
{
    NvtxRange nvtx_range("gblu_refactorize_multi");
    if (nh < 1 || !hs || !Ax_dev) return fail(GBLU_ERR_INVALID_INPUT, "multi: nh >= 1 and non-null arrays");
    for (int32_t i = 0; i < nh; i++) {
        CK(check_handle(hs[i]));
        if (!hs[i]->factorized) return fail(GBLU_ERR_NOT_FACTORIZED, "multi: handle %d is not factorized", i);
        if (!Ax_dev[i]) return fail(GBLU_ERR_INVALID_INPUT, "multi: null values for handle %d", i);
        if (hs[i]->device != hs[0]->device) return fail(GBLU_ERR_INVALID_INPUT, "multi: handles on different devices");
        if (repivoted) repivoted[i] = 0;
    }
    {
        std::vector<const void *> u(hs, hs + nh);
        std::sort(u.begin(), u.end());
        if (std::adjacent_find(u.begin(), u.end()) != u.end())
            return fail(GBLU_ERR_INVALID_INPUT, "multi: a handle appears twice");
    }
    gblu_ctx *h0 = hs[0];
    DeviceGuard g(h0->device);
    cudaStream_t st = (cudaStream_t)stream;
    // one epoch for every set (epochs only grow, so old flags never match)
    int32_t ep = 0;
    for (int32_t i = 0; i < nh; i++) ep = std::max(ep, hs[i]->epoch);
    ep++;
    // merged ticket order: every set's tasks in its own (topological) order,
    // interleaved so that all sets advance at the same relative pace
    std::vector<std::pair<const void *, uint64_t>> key(nh);
    for (int32_t i = 0; i < nh; i++) key[i] = {hs[i], hs[i]->struct_version};
    if (key != h0->morder_key || !h0->morder.p) {
        std::vector<int64_t> T(nh);
        int64_t total = 0;
        for (int32_t i = 0; i < nh; i++) total += (T[i] = (int64_t)hs[i]->W.task_ptr.size() - 1);
        if (total > INT32_MAX) return fail(GBLU_ERR_INVALID_INPUT, "multi: too many tasks");
        std::vector<SetTask> ord;
        ord.reserve(total);
        using Item = std::pair<double, int32_t>;   // (next key, set)
        std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
        std::vector<int64_t> next(nh, 0);
        for (int32_t i = 0; i < nh; i++)
            if (T[i] > 0) pq.push({0.5 / (double)T[i], i});
        while (!pq.empty()) {
            const int32_t i = pq.top().second;
            pq.pop();
            ord.push_back({i, (int32_t)next[i]});
            if (++next[i] < T[i]) pq.push({((double)next[i] + 0.5) / (double)T[i], i});
        }
        CK(upload(h0, h0->morder, ord, st));
        h0->morder_key = key;
        h0->morder_n = total;
    }
    CK(ensure(h0, h0->bargs, (size_t)nh));
    CK(ensure(h0, h0->bticket, 1));
    h0->bargs_host.resize(nh);
    for (int32_t i = 0; i < nh; i++) {
        gblu_ctx *h = hs[i];
        h->epoch = ep;
        h->n_refactor++;
        RefactorArgs a = refactor_args(h, Ax_dev[i]);
        a.dense_p = INT_MAX;   // the dense tail is not used in batches
        h0->bargs_host[i] = a;
    }
    CU(cudaMemcpyAsync(h0->bargs.p, h0->bargs_host.data(), sizeof(RefactorArgs) * nh, cudaMemcpyHostToDevice, st));
    {
        gblu_ctx *h = h0;   // the launch is counted on the leading handle
        bool pull = false;
        for (int32_t i = 0; i < nh; i++) pull = pull || hs[i]->pull_slots > 0;
        KL(launch_refactor_multi(h0->bargs.p, h0->bargs_host[0], nh, h0->morder.p, (int)h0->morder_n, pgrid(h0, h0->batch_blocks_per_sm),
                                 ep, h0->bticket.p, st, pull));
        h->launches++;   // the control-block reset kernel
    }
    for (int32_t i = 0; i < nh; i++)
        CU(cudaMemcpyAsync(hs[i]->hctl, hs[i]->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    // sets whose check failed restart alone (Section IV-C)
    for (int32_t i = 0; i < nh; i++) {
        gblu_ctx *h = hs[i];
        if (h->hctl->status != 0) {
            h->factorized = false;
            return fail(h->hctl->status, "multi: handle %d: device status %d", i, h->hctl->status);
        }
        h->last_first_bad = h->hctl->interrupted ? h->hctl->first_bad : -1;
        if (!h->hctl->interrupted) continue;
        h->n_repivot++;
        const int rc = run_restart(h, Ax_dev[i], st);
        if (rc != GBLU_OK) {
            h->factorized = false;
            return rc;
        }
        if (repivoted) repivoted[i] = 1;
    }
    return GBLU_OK;
}

int gblu_solve_multi(int32_t nh, gblu_handle *hs, const double *const *b_dev, double *const *x_dev, void *stream)
{
    NvtxRange nvtx_range("gblu_solve_multi");
    if (nh < 1 || !hs || !b_dev || !x_dev) return fail(GBLU_ERR_INVALID_INPUT, "multi: nh >= 1 and non-null arrays");
    cudaStream_t st = (cudaStream_t)stream;
    // handles whose solve is all sparse row blocks go into one launch per
    // triangle; the others (trailing dense pieces) are solved one by one
    std::vector<gblu_ctx *> fused;
    std::vector<int32_t> fi, alone;
    for (int32_t i = 0; i < nh; i++) {
        gblu_ctx *h = hs[i];
        CK(check_handle(h));
        if (!h->factorized) return fail(GBLU_ERR_NOT_FACTORIZED, "multi: handle %d is not factorized", i);
        if (!b_dev[i] || !x_dev[i]) return fail(GBLU_ERR_INVALID_INPUT, "multi: null vector for handle %d", i);
        if (h->device != hs[0]->device) return fail(GBLU_ERR_INVALID_INPUT, "multi: handles on different devices");
        if (h->W.lp0 < h->S.n || h->W.up0 < h->S.n) {
            alone.push_back(i);
        } else {
            fused.push_back(h);
            fi.push_back(i);
        }
    }
    {
        std::vector<const void *> u(hs, hs + nh);
        std::sort(u.begin(), u.end());
        if (std::adjacent_find(u.begin(), u.end()) != u.end())
            return fail(GBLU_ERR_INVALID_INPUT, "multi: a handle appears twice");
    }
    DeviceGuard g(hs[0]->device);
    // handles with trailing dense pieces solve on their own streams, forked
    // from `stream` and joined back, overlapping the fused launch (each
    // solve is latency-bound and uses a fraction of the device)
    EventList events;
    std::vector<cudaEvent_t> joins;
    if (!alone.empty()) {
        cudaEvent_t fork;
        CK(events.record(st, &fork));
        for (int32_t i : alone) {
            gblu_ctx *h = hs[i];
            if (!h->aux) CU(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
            CU(cudaStreamWaitEvent(h->aux, fork, 0));
            CK(gblu_solve(h, b_dev[i], x_dev[i], h->aux));
            cudaEvent_t j;
            CK(events.record(h->aux, &j));
            joins.push_back(j);
        }
    }
    // `stream` waits for the forked solves (an error before this leaves
    // them unjoined; the call then reports it)
    auto join = [&]() -> int {
        for (cudaEvent_t j : joins) CU(cudaStreamWaitEvent(st, j, 0));
        return GBLU_OK;
    };
    const int32_t nf = (int32_t)fused.size();
    if (nf == 0) return join();
    gblu_ctx *h0 = fused[0];
    std::vector<std::pair<const void *, uint64_t>> key(nf);
    for (int32_t i = 0; i < nf; i++) key[i] = {fused[i], fused[i]->struct_version};
    if (key != h0->msolve_key || !h0->mlorder.p) {
        // every set's rows in its own ticket order, interleaved by relative progress
        auto merge = [&](bool lower, DBuf<SetTask> &out, int64_t &count) -> int {
            std::vector<int64_t> T(nf);
            int64_t total = 0;
            for (int32_t i = 0; i < nf; i++)
                total += (T[i] = (int64_t)(lower ? fused[i]->W.lsv_tick.size() : fused[i]->W.usv_tick.size()));
            if (total > INT32_MAX) return fail(GBLU_ERR_INVALID_INPUT, "multi: too many rows");
            std::vector<SetTask> ord;
            ord.reserve(total);
            using Item = std::pair<double, int32_t>;
            std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
            std::vector<int64_t> next(nf, 0);
            for (int32_t i = 0; i < nf; i++)
                if (T[i] > 0) pq.push({0.5 / (double)T[i], i});
            while (!pq.empty()) {
                const int32_t i = pq.top().second;
                pq.pop();
                ord.push_back({i, (int32_t)next[i]});
                if (++next[i] < T[i]) pq.push({((double)next[i] + 0.5) / (double)T[i], i});
            }
            CK(upload(h0, out, ord, st));
            count = total;
            return GBLU_OK;
        };
        CK(merge(true, h0->mlorder, h0->mlorder_n));
        CK(merge(false, h0->muorder, h0->muorder_n));
        h0->msolve_key = key;
    }
    h0->margs_host.resize(2 * (size_t)nf);
    int32_t max_n = 0;
    for (int32_t i = 0; i < nf; i++) {
        gblu_ctx *h = fused[i];
        SolveArgs a = solve_args(h, h->vals.p, b_dev[fi[i]], x_dev[fi[i]]);
        SolveArgs lo = a, up = a;
        lo.bs = h->lbs.p;
        lo.rb = h->lrb.p;
        lo.ext = h->ext_l.p;
        lo.rows = h->lsv_tick.p;
        lo.nrows = (int32_t)h->W.lsv_tick.size();
        up.bs = h->ubs.p;
        up.rb = h->urb.p;
        up.ext = h->ext_u.p;
        up.rows = h->usv_tick.p;
        up.nrows = (int32_t)h->W.usv_tick.size();
        h0->margs_host[i] = lo;
        h0->margs_host[nf + i] = up;
        max_n = std::max(max_n, h->S.n);
    }
    CK(ensure(h0, h0->margs, 2 * (size_t)nf));
    CK(ensure(h0, h0->mticket, 2));
    CU(cudaMemcpyAsync(h0->margs.p, h0->margs_host.data(), sizeof(SolveArgs) * 2 * nf, cudaMemcpyHostToDevice, st));
    {
        gblu_ctx *h = h0;
        KL(launch_solve_multi(h0->margs.p, h0->margs.p + nf, nf, max_n, h0->mlorder.p, (int)h0->mlorder_n,
                              h0->muorder.p, (int)h0->muorder_n, h0->solve_grid, h0->mticket.p, st));
        h->launches += 2;   // three kernels
    }
    // the argument block is read by the kernels: keep the host copy unchanged
    // until they have been issued (the copy above is stream-ordered)
    return join();
}

// capture [epoch -> control block, checked re-factorization, control block
// -> host, solve] on the handle's staging buffers into one graph
static int capture_step(gblu_ctx *h)
{
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    if (!h->gstream) CU(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
    if (!h->epoch_host) CU(cudaMallocHost((void **)&h->epoch_host, sizeof(int32_t)));
    cudaStream_t gs = h->gstream;
    const long long l0 = h->launches;
    CU(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
    int rc = GBLU_OK;
    if (cudaMemcpyAsync(&h->ctl->epoch, h->epoch_host, sizeof(int32_t), cudaMemcpyHostToDevice, gs) != cudaSuccess)
        rc = fail(GBLU_ERR_CUDA, "graph capture: epoch copy failed");
    if (rc == GBLU_OK) rc = issue_refactor(h, h->stage_ax.p, gs, -1);
    if (rc == GBLU_OK &&
        cudaMemcpyAsync(h->hctl, h->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, gs) != cudaSuccess)
        rc = fail(GBLU_ERR_CUDA, "graph capture: status copy failed");
    if (rc == GBLU_OK) rc = solve_values(h, h->vals.p, 0, h->stage_b.p, 0, h->stage_x.p, 0, 1, gs);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(gs, &graph);
    h->glaunches = h->launches - l0;
    h->launches = l0;   // counted per replay instead
    if (rc != GBLU_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail(GBLU_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) {
        h->gexec = nullptr;
        return fail(GBLU_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e2));
    }
    h->gversion = h->struct_version;
    h->glayout = h->layout_version;
    return GBLU_OK;
}

int gblu_step(gblu_handle h, const double *Ax_dev, const double *b_dev, double *x_dev, void *stream,
              int32_t *repivoted)
{
    NvtxRange nvtx_range("gblu_step");
    CK(check_handle(h));
    h->last_repivot = false;
    if (repivoted) *repivoted = 0;
    if (!h->factorized) return fail(GBLU_ERR_NOT_FACTORIZED, "gblu_factorize has not succeeded");
    if (!Ax_dev || !b_dev || !x_dev) return fail(GBLU_ERR_INVALID_INPUT, "null vector");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t n = h->S.n;
    const size_t nnz = h->P.Ai.size();
    CK(ensure(h, h->stage_ax, nnz));
    CK(ensure(h, h->stage_b, n));
    CK(ensure(h, h->stage_x, n));
    if (!h->gexec || h->gversion != h->struct_version || h->glayout != h->layout_version) CK(capture_step(h));
    CU(cudaMemcpyAsync(h->stage_ax.p, Ax_dev, nnz * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(h->stage_b.p, b_dev, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // the previous call ended with a synchronization, so the pinned epoch
    // word is free to change
    h->epoch++;
    h->n_refactor++;
    *h->epoch_host = h->epoch;
    CU(cudaGraphLaunch(h->gexec, st));
    h->launches += h->glaunches;
    CU(cudaMemcpyAsync(x_dev, h->stage_x.p, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CU(cudaStreamSynchronize(st));
    CK(status_code(h));
    h->last_first_bad = h->hctl->interrupted ? h->hctl->first_bad : -1;
    if (!h->hctl->interrupted) return GBLU_OK;
    // the check failed: the solve of the replay is void; restart, solve again
    h->n_repivot++;
    int rc = run_restart(h, h->stage_ax.p, st);
    if (rc != GBLU_OK) {
        h->factorized = false;
        return rc;
    }
    CK(solve_values(h, h->vals.p, 0, b_dev, 0, x_dev, 0, 1, st));
    if (repivoted) *repivoted = 1;
    h->last_repivot = true;
    return GBLU_REPIVOTED;
}

// capture [flag reset, batch refactor (cluster levels, pipeline), control
// blocks -> pinned host, batch solve] for the given buffers into one graph.
// The flags are cleared inside the graph, so every replay uses epoch 1.
static int capture_step_batch(gblu_ctx *h, int32_t nsets, const double *Ax_dev, int64_t ax_stride,
                              double *LUx_dev, int64_t lu_stride, const double *b_dev, int64_t b_stride,
                              double *x_dev, int64_t x_stride)
{
    if (h->bgexec) {
        cudaGraphExecDestroy(h->bgexec);
        h->bgexec = nullptr;
    }
    const int32_t n = h->S.n;
    CK(ensure(h, h->bgargs, (size_t)nsets));
    if (h->bgctl_cap < nsets) {
        if (h->bgctl_host) cudaFreeHost(h->bgctl_host);
        h->bgctl_host = nullptr;
        h->bgctl_cap = 0;
        CU(cudaMallocHost((void **)&h->bgctl_host, sizeof(DevCtl) * (size_t)nsets));
        h->bgctl_cap = nsets;
    }
    if (!h->gstream) CU(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
    const RefactorArgs base = refactor_args(h, nullptr);
    std::vector<RefactorArgs> args(nsets, base);
    for (int32_t s = 0; s < nsets; s++) {
        args[s].Ax = Ax_dev + s * ax_stride;
        args[s].LUx = LUx_dev + s * lu_stride;
        args[s].finish = h->bfinish.p + (size_t)s * n;
        args[s].ctl = h->bctl.p + s;
        args[s].dense_p = INT_MAX;   // the dense tail is not used in batches
    }
    cudaStream_t gs = h->gstream;
    CU(cudaMemcpyAsync(h->bgargs.p, args.data(), sizeof(RefactorArgs) * nsets, cudaMemcpyHostToDevice, gs));
    CU(cudaStreamSynchronize(gs));
    const long long l0 = h->launches;
    CU(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
    int rc = GBLU_OK;
    auto step = [&]() -> int {
        CU(cudaMemsetAsync(h->bfinish.p, 0, sizeof(int32_t) * (size_t)nsets * n, gs));
        KL(launch_begin_batch(h->bctl.p, nsets, h->bticket.p, gs));
        RefactorArgs a0 = base;
        const std::vector<int32_t> &ltp = h->W.level_task_ptr;
        const int32_t div = h->W.div_level;
        for (int32_t l = 0; l < div; l++) {
            a0.task_begin = ltp[l];
            a0.ntasks = ltp[l + 1] - ltp[l];
            KL(launch_refactor_batch(h->bgargs.p, a0, nsets, false, 0, 1, h->bticket.p, gs, nsets));
        }
        const int32_t ntask = (int32_t)h->W.task_ptr.size() - 1;
        if (ltp[div] < ntask) {
            a0.task_begin = ltp[div];
            a0.ntasks = ntask - ltp[div];
            KL(launch_refactor_batch(h->bgargs.p, a0, nsets, true, pgrid(h, h->batch_blocks_per_sm), 1, h->bticket.p, gs,
                                     batch_group(h, nsets)));
        }
        CU(cudaMemcpyAsync(h->bgctl_host, h->bctl.p, sizeof(DevCtl) * nsets, cudaMemcpyDeviceToHost, gs));
        return solve_values(h, LUx_dev, lu_stride, b_dev, b_stride, x_dev, x_stride, nsets, gs);
    };
    rc = step();
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(gs, &graph);
    h->bglaunches = h->launches - l0;
    h->launches = l0;   // counted per replay instead
    if (rc != GBLU_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail(GBLU_ERR_CUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(&h->bgexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) {
        h->bgexec = nullptr;
        return fail(GBLU_ERR_CUDA, "batch graph instantiation failed: %s", cudaGetErrorString(e2));
    }
    h->bgversion = h->struct_version;
    h->bglayout = h->layout_version;
    return GBLU_OK;
}

int gblu_step_batch(gblu_handle h, int32_t nsets, const double *Ax_dev, int64_t ax_stride, double *LUx_dev,
                    int64_t lu_stride, const double *b_dev, int64_t b_stride, double *x_dev, int64_t x_stride,
                    int32_t *failed, int32_t *n_failed, void *stream)
{
    NvtxRange nvtx_range("gblu_step_batch");
    CK(check_handle(h));
    if (n_failed) *n_failed = 0;
    if (!h->factorized) return fail(GBLU_ERR_NOT_FACTORIZED, "gblu_factorize has not succeeded");
    const int32_t n = h->S.n;
    if (nsets < 1 || !b_dev || !x_dev || b_stride < n || x_stride < n)
        return fail(GBLU_ERR_INVALID_INPUT, "step batch: nsets >= 1, non-null vectors, strides >= n");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const std::vector<int64_t> key = {nsets, (int64_t)(uintptr_t)Ax_dev, ax_stride, (int64_t)(uintptr_t)LUx_dev,
                                      lu_stride, (int64_t)(uintptr_t)b_dev, b_stride, (int64_t)(uintptr_t)x_dev,
                                      x_stride};
    if (!h->bgexec || key != h->bgkey || h->bgversion != h->struct_version || h->bglayout != h->layout_version) {
        // first call with these buffers: run eagerly (this sizes every
        // buffer the graph uses), then capture for the next calls
        CK(gblu_refactorize_batch(h, nsets, Ax_dev, ax_stride, LUx_dev, lu_stride, failed, n_failed, stream));
        CK(gblu_solve_batch(h, nsets, LUx_dev, lu_stride, b_dev, b_stride, x_dev, x_stride, stream));
        CU(cudaStreamSynchronize(st));
        h->bgkey.clear();
        CK(capture_step_batch(h, nsets, Ax_dev, ax_stride, LUx_dev, lu_stride, b_dev, b_stride, x_dev, x_stride));
        h->bgkey = key;
        return GBLU_OK;
    }
    h->n_refactor += nsets;
    CU(cudaGraphLaunch(h->bgexec, st));
    h->launches += h->bglaunches;
    CU(cudaStreamSynchronize(st));
    int32_t nf = 0;
    for (int32_t s = 0; s < nsets; s++) {
        const DevCtl &c = h->bgctl_host[s];
        if (c.status != 0) return fail(c.status, "batch set %d: device status %d (wait %d at column %d)", s,
                                       c.status, c.where, c.where_k);
        if (failed) failed[s] = c.interrupted ? 1 : 0;
        nf += c.interrupted ? 1 : 0;
    }
    if (n_failed) *n_failed = nf;
    return GBLU_OK;
}

int gblu_gather_scale(int64_t m, const int32_t *src_dev, const double *scale_dev, const double *in_dev,
                      double *out_dev, void *stream)
{
    if (m < 0 || !in_dev || !out_dev) return fail(GBLU_ERR_INVALID_INPUT, "gather_scale: m >= 0 and non-null vectors");
    if (in_dev == out_dev && src_dev) return fail(GBLU_ERR_INVALID_INPUT, "gather_scale: a gather cannot be in place");
    const int e = launch_gather_scale(m, src_dev, scale_dev, in_dev, out_dev, stream);
    if (e != 0) return fail(GBLU_ERR_CUDA, "gather_scale launch failed: %s", cudaGetErrorString((cudaError_t)e));
    return GBLU_OK;
}

int gblu_get_opts(gblu_handle h, gblu_opts *o)
{
    if (!h || !o) return fail(GBLU_ERR_INVALID_INPUT, "null pointer");
    *o = h->opts;
    return GBLU_OK;
}

int gblu_set_opts(gblu_handle h, const gblu_opts *o, void *stream)
{
    if (!h || !o) return fail(GBLU_ERR_INVALID_INPUT, "null pointer");
    if (!opts_valid(*o)) return fail(GBLU_ERR_INVALID_INPUT, "invalid options");
    DeviceGuard g(h->device);
    h->opts = *o;
    if (!h->factorized) return GBLU_OK;
    // same factor structure and values; the schedule follows the new options
    Structure S = h->S;
    return install_structure(h, std::move(S), nullptr, (cudaStream_t)stream);
}

int gblu_autotune(gblu_handle h, const double *Ax_dev, const double *b_dev, double *x_dev, int32_t reps,
                  void *stream, gblu_opts *chosen, double *refactor_ms, double *solve_ms)
{
    CK(check_handle(h));
    if (!h->factorized) return fail(GBLU_ERR_NOT_FACTORIZED, "gblu_factorize has not succeeded");
    if (!Ax_dev || !b_dev || !x_dev || reps < 1) return fail(GBLU_ERR_INVALID_INPUT, "null vector or reps < 1");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1, e2;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    CU(cudaEventCreate(&e2));
    // median refactor and solve times of the current options (one untimed run first)
    auto measure = [&](double &tr, double &ts) -> int {
        std::vector<float> a, b;
        for (int32_t r = -1; r < reps; r++) {
            int intr = 0;
            CU(cudaEventRecord(e0, st));
            CK(run_refactor(h, Ax_dev, st, &intr));
            if (intr) {
                h->n_repivot++;
                CK(run_restart(h, Ax_dev, st));
            }
            CU(cudaEventRecord(e1, st));
            CK(solve_values(h, h->vals.p, 0, b_dev, 0, x_dev, 0, 1, st));
            CU(cudaEventRecord(e2, st));
            CU(cudaEventSynchronize(e2));
            float m1 = 0, m2 = 0;
            CU(cudaEventElapsedTime(&m1, e0, e1));
            CU(cudaEventElapsedTime(&m2, e1, e2));
            if (r >= 0) {
                a.push_back(m1);
                b.push_back(m2);
            }
        }
        std::sort(a.begin(), a.end());
        std::sort(b.begin(), b.end());
        tr = a[a.size() / 2];
        ts = b[b.size() / 2];
        return GBLU_OK;
    };
    gblu_opts best = h->opts;
    double br = 0, bs = 0;
    int rc = measure(br, bs);
    // the dividing level of the re-factorization (Section IV-B: alpha), then
    // the trailing-block rule of the solve (Section V-A: P0 and the slices)
    const double alphas[] = {0.25, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0};
    for (double al : alphas) {
        if (rc != GBLU_OK) break;
        if (al == best.alpha) continue;
        gblu_opts o = best;
        o.alpha = al;
        double tr = 0, ts = 0;
        if ((rc = gblu_set_opts(h, &o, stream)) != GBLU_OK || (rc = measure(tr, ts)) != GBLU_OK) break;
        if (tr < br) {
            best = o;
            br = tr;
            bs = ts;
        }
    }
    // the warp assignment: the longest column one warp computes (Section
    // IV-B's task granularity), by re-factorization time
    const int wcols[] = {256, 512, kRefCapShort};
    for (int wc : wcols) {
        if (rc != GBLU_OK) break;
        if (wc == best.warp_column_max) continue;
        gblu_opts o = best;
        o.warp_column_max = wc;
        double tr = 0, ts = 0;
        if ((rc = gblu_set_opts(h, &o, stream)) != GBLU_OK || (rc = measure(tr, ts)) != GBLU_OK) break;
        if (tr < br) {
            best = o;
            br = tr;
            bs = ts;
        }
    }
    const double dens[] = {0.0, 0.3, 0.5, 0.7, 0.9};
    // slices only switch the trailing block on (> 0) or off (0): the
    // kernels cut it into 32-row slices whatever the count
    const int slices[] = {0, 8};
    for (double dd : dens) {
        for (int m : slices) {
            if (rc != GBLU_OK) break;
            if (dd == best.solve_dense_density && m == best.solve_slices) continue;
            gblu_opts o = best;
            o.solve_dense_density = dd;
            o.solve_slices = m;
            double tr = 0, ts = 0;
            if ((rc = gblu_set_opts(h, &o, stream)) != GBLU_OK || (rc = measure(tr, ts)) != GBLU_OK) break;
            if (ts < bs) {
                best = o;
                bs = ts;
            }
        }
    }
    for (int per : {0, 1, 2, 4}) {   // resident warps of the sync-free solves
        if (rc != GBLU_OK || per == best.solve_ctas_per_sm) continue;
        gblu_opts o = best;
        o.solve_ctas_per_sm = per;
        double tr = 0, ts = 0;
        if ((rc = gblu_set_opts(h, &o, stream)) != GBLU_OK || (rc = measure(tr, ts)) != GBLU_OK) break;
        if (ts < bs) {
            best = o;
            bs = ts;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    if (rc != GBLU_OK) return rc;
    CK(gblu_set_opts(h, &best, stream));
    if (chosen) *chosen = best;
    if (refactor_ms) *refactor_ms = br;
    if (solve_ms) *solve_ms = bs;
    return GBLU_OK;
}

int gblu_refactorize_f32(gblu_handle h, const double *Ax_dev, void *stream, int32_t *check_failed)
{
    NvtxRange nvtx_range("gblu_refactorize_f32");
    CK(check_handle(h));
    if (check_failed) *check_failed = 0;
    if (!h->factorized) return fail(GBLU_ERR_NOT_FACTORIZED, "gblu_factorize has not succeeded");
    if (!Ax_dev) return fail(GBLU_ERR_INVALID_INPUT, "null Ax_dev");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    CK(ensure(h, h->vals32, (size_t)h->S.nnz()));
    h->epoch++;
    h->n_refactor++;
    KL(launch_begin_refactor(h->ctl, st));
    const RefactorArgs d = refactor_args(h, Ax_dev);
    RefactorArgsT<float> a{};
    a.Ap = d.Ap; a.Q = d.Q; a.amap = d.amap; a.Ax = d.Ax; a.LUp = d.LUp; a.LUi = d.LUi; a.nU = d.nU;
    a.chain = d.chain; a.dense_p = INT_MAX; a.dense_s0 = nullptr; a.S = nullptr; a.dense_ld = 0;
    a.LUx = h->vals32.p; a.finish = d.finish; a.task_ptr = d.task_ptr; a.task_cols = d.task_cols;
    a.cap_short = d.cap_short; a.cap_long = d.cap_long; a.eps = d.eps; a.spin_limit = d.spin_limit;
    a.ctl = d.ctl;
    const std::vector<int32_t> &ltp = h->W.level_task_ptr;
    const int32_t div = h->W.div_level;
    for (int32_t l = 0; l < div; l++) {
        a.task_begin = ltp[l];
        a.ntasks = ltp[l + 1] - ltp[l];
        KL(launch_refactor_tasks_f32(a, false, 0, h->epoch, st));
    }
    const int32_t ntask = (int32_t)h->W.task_ptr.size() - 1;
    if (ltp[div] < ntask) {
        a.task_begin = ltp[div];
        a.ntasks = ntask - ltp[div];
        KL(launch_refactor_tasks_f32(a, true, pgrid(h, h->ref32_blocks_per_sm), h->epoch, st));
    }
    // the pivots in double: a pivot that single precision cannot place
    // clearly on the passing side of the threshold fails here, and the
    // double-precision re-factorization then decides
    KL(launch_f32_verify(h->S.n, h->LUp.p, h->LUi.p, h->nU.p, h->vals32.p, h->Lrp.p, h->Lcol.p, h->Lslot.p,
                         h->opts.pivot_tol, h->ctl, h->sm_count * 8, st));
    CK(read_ctl(h, st));
    CK(status_code(h));
    h->f32_valid = !h->hctl->interrupted;
    h->f32_widened = false;
    h->last_first_bad = h->hctl->interrupted ? h->hctl->first_bad : -1;
    if (check_failed) *check_failed = h->hctl->interrupted ? 1 : 0;
    return GBLU_OK;
}

int gblu_solve_refined(gblu_handle h, const double *Ax_dev, const double *b_dev, double *x_dev, double tol,
                       int32_t max_iter, void *stream, int32_t *iters, double *berr)
{
    NvtxRange nvtx_range("gblu_solve_refined");
    CK(check_handle(h));
    if (iters) *iters = 0;
    if (!h->factorized) return fail(GBLU_ERR_NOT_FACTORIZED, "gblu_factorize has not succeeded");
    if (!Ax_dev || !b_dev || !x_dev || !(tol >= 0.0) || max_iter < 0)
        return fail(GBLU_ERR_INVALID_INPUT, "null vector, negative tolerance or iteration limit");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t n = h->S.n;
    const size_t nnz = (size_t)h->S.nnz();
    CK(ensure(h, h->ir_r, (size_t)n));
    CK(ensure(h, h->ir_d, (size_t)n));
    CK(ensure(h, h->ir_out, 4));
    if (!h->ir_host) CU(cudaMallocHost((void **)&h->ir_host, 4 * sizeof(double)));
    // backward error ||b - A x||inf / (||A||inf ||x||inf); r = b - A x kept in ir_r
    auto residual = [&](const double *x, double *out_host) -> int {
        KL(launch_residual(h->P.n, h->Arp.p, h->Acol.p, h->Aslot.p, Ax_dev, b_dev, x, h->ir_out.p,
                           h->partial.p, h->res_blocks, st, h->ir_r.p));
        CU(cudaMemcpyAsync(h->ir_host, h->ir_out.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        *out_host = h->ir_host[0];
        return GBLU_OK;
    };
    double e = 0.0;
    int32_t it = 0;
    bool converged = false;
    if (h->f32_valid) {
        if (!h->f32_widened) {
            CK(ensure(h, h->vals_w, nnz));
            KL(launch_widen(h->vals32.p, h->vals_w.p, (int64_t)nnz, st));
            h->f32_widened = true;
        }
        CK(solve_values(h, h->vals_w.p, 0, b_dev, 0, x_dev, 0, 1, st));
        CK(residual(x_dev, &e));
        double prev = e;
        while (!(e <= tol) && it < max_iter) {
            CK(solve_values(h, h->vals_w.p, 0, h->ir_r.p, 0, h->ir_d.p, 0, 1, st));   // A d = r
            KL(launch_axpy(x_dev, h->ir_d.p, n, st));
            it++;
            CK(residual(x_dev, &e));
            if (!(e <= 0.5 * prev)) break;   // refinement stalls
            prev = e;
        }
        converged = e <= tol;
    }
    if (!converged) {   // the FP64 re-factorization (with its restart) and solve
        int interrupted = 0;
        int rc = run_refactor(h, Ax_dev, st, &interrupted);
        if (rc == GBLU_OK && interrupted) {
            h->n_repivot++;
            rc = run_restart(h, Ax_dev, st);
        }
        if (rc != GBLU_OK) {
            h->factorized = false;
            return rc;
        }
        CK(solve_values(h, h->vals.p, 0, b_dev, 0, x_dev, 0, 1, st));
        CK(residual(x_dev, &e));
        it = -1;
    }
    if (iters) *iters = it;
    if (berr) *berr = e;
    return GBLU_OK;
}

int gblu_step_host(gblu_handle h, const double *Ax_host, const double *b_host, double *x_host,
                   void *stream, int32_t *repivoted)
{
    CK(check_handle(h));
    if (repivoted) *repivoted = 0;
    if (!Ax_host || !b_host || !x_host) return fail(GBLU_ERR_INVALID_INPUT, "null host pointer");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nnz = h->P.Ai.size(), n = (size_t)h->P.n;
    CK(ensure(h, h->stage_ax, nnz));
    CK(ensure(h, h->stage_b, n));
    CK(ensure(h, h->stage_x, n));
    CU(cudaMemcpyAsync(h->stage_ax.p, Ax_host, nnz * sizeof(double), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(h->stage_b.p, b_host, n * sizeof(double), cudaMemcpyHostToDevice, st));
    const int rc = gblu_refactorize(h, h->stage_ax.p, stream, repivoted);
    if (rc < 0) return rc;
    CK(gblu_solve(h, h->stage_b.p, h->stage_x.p, stream));
    CU(cudaMemcpyAsync(x_host, h->stage_x.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return rc;
}

int gblu_residual(gblu_handle h, const double *Ax_dev, const double *b_dev, const double *x_dev,
                  double *out_dev, void *stream)
{
    CK(check_handle(h));
    if (!Ax_dev || !b_dev || !x_dev || !out_dev) return fail(GBLU_ERR_INVALID_INPUT, "null pointer");
    DeviceGuard g(h->device);
    KL(launch_residual(h->P.n, h->Arp.p, h->Acol.p, h->Aslot.p, Ax_dev, b_dev, x_dev, out_dev,
                       h->partial.p, h->res_blocks, (cudaStream_t)stream));
    h->launches++;  // the residual is two kernels
    return GBLU_OK;
}

int gblu_get_stats(gblu_handle h, gblu_stats *s)
{
    if (!h || !s) return fail(GBLU_ERR_INVALID_INPUT, "null pointer");
    std::memset(s, 0, sizeof(*s));
    s->n = h->P.n;
    s->nnz_a = (int64_t)h->P.Ai.size();
    s->etree_height = h->P.cetree_height;
    s->n_refactor = h->n_refactor;
    s->n_repivot = h->n_repivot;
    s->n_restart_cols = h->n_restart_cols;
    s->last_first_bad = h->last_first_bad;
    s->device_bytes = (int64_t)h->device_bytes;
    s->kernel_launches = h->launches;
    s->dense_rows = h->W.dense_m;
    s->tail_kernel_ms = h->t_tail[0];
    s->tail_repack_ms = h->t_tail[1];
    s->tail_schedule_ms = h->t_tail[2];
    s->tail_upload_ms = h->t_tail[3];
    s->tail_passes = h->tail_passes;
    s->first_mode = h->first_mode;
    s->first_symbolic_ms = h->t_first_symbolic;
    s->wide_cols = h->pull_slots > 0 ? h->W.pull_cols : 0;
    s->repredictions = h->repredictions;
    if (h->factorized) {
        int64_t nu = 0;
        for (int32_t v : h->S.nU) nu += v;
        s->nnz_u = nu;
        s->nnz_l = h->S.nnz() - nu;
        s->flops = h->W.flops;
        s->n_levels = h->W.n_levels;
        s->div_level = h->W.div_level;
        s->n_solve_levels_l = h->W.lsv_levels;
        s->n_solve_levels_u = h->W.usv_levels;
        s->solve_p0_l = h->W.lp0;
        s->solve_p0_u = h->W.up0;
        s->solve_slices_l = h->W.lcut.empty() ? 0 : (int32_t)h->W.lcut.size() - 1;
        s->solve_slices_u = h->W.ucut.empty() ? 0 : (int32_t)h->W.ucut.size() - 1;
    }
    return GBLU_OK;
}

int gblu_export_factors(gblu_handle h, int64_t *Lp, int32_t *Li, double *Lx, int64_t *Up,
                        int32_t *Ui, double *Ux, int32_t *piv, int32_t *q)
{
    CK(check_handle(h));
    if (!h->factorized) return fail(GBLU_ERR_NOT_FACTORIZED, "no valid factorization");
    DeviceGuard g(h->device);
    const Structure &S = h->S;
    const int32_t n = S.n;
    std::vector<double> v(S.nnz());
    CU(cudaDeviceSynchronize());
    if (!v.empty()) CU(cudaMemcpy(v.data(), h->vals.p, v.size() * sizeof(double), cudaMemcpyDeviceToHost));
    int64_t lo = 0, uo = 0;
    if (Lp) Lp[0] = 0;
    if (Up) Up[0] = 0;
    for (int32_t k = 0; k < n; k++) {
        for (int64_t e = S.LUp[k]; e < S.LUp[k + 1]; e++) {
            if (e - S.LUp[k] < S.nU[k]) {
                if (Ui) Ui[uo] = S.LUi[e];
                if (Ux) Ux[uo] = v[e];
                uo++;
            } else {
                if (Li) Li[lo] = S.LUi[e];
                if (Lx) Lx[lo] = v[e];
                lo++;
            }
        }
        if (Lp) Lp[k + 1] = lo;
        if (Up) Up[k + 1] = uo;
    }
    if (piv) std::memcpy(piv, S.piv.data(), sizeof(int32_t) * n);
    if (q) std::memcpy(q, h->P.Q.data(), sizeof(int32_t) * n);
    return GBLU_OK;
}

}  // extern "C"
