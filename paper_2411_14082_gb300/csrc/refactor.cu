// Checked re-factorization on a fixed pattern (Section IV-B, Algorithms 3
// and 4), CSC left-looking form.
//
// Column k's pattern (step numbers, sorted: U rows, diagonal k, L rows) is
// the index set of its work vector x.  x = A(:,Q[k]) is scattered through
// amap; then for every dependency j (the U rows above the diagonal, in
// ascending order, which is a topological order)
//     x(rows of L(:,j)) -= x(j) * L(:,j);
// then the pivot check |x(k)| >= eps * max|x(L rows)| and x(k) != 0, and
// the stores U(:,k) = x(U rows), L(:,k) = x(L rows) / x(k).
//
// Work is handed out as tasks (built on the host in level order): a task is
// one long column (all 8 warps of a CTA, work vector of up to 5,120 entries
// in shared memory), two medium columns (4 warps and up to 2,560 entries
// each, synchronized by named barriers), or up to 8 short columns (one per
// warp).  The
// slot of an L(:,j) row inside column k comes from a binary search in the
// sorted pattern over [t+1+i, t+(r-j)] (t = slot of j, i = index of the row
// inside L(:,j)); the interval is exact inside dense runs, so dense parts
// need no search steps.  L(:,k) is stored as x * (1 / x(k)).
//
// Two schedules (Section IV-B): cluster mode = one launch per level with no
// waits; pipeline mode = one persistent launch whose CTAs take tasks by an
// atomic ticket and wait on per-column ready flags (epochs) before using a
// dependency.  A failing pivot sets `interrupted` (Algorithm 3 line 9 /
// Algorithm 4 line 11); waiting CTAs poll it and leave.  Every wait is
// bounded by spin_limit iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <type_traits>

#include "device_util.cuh"
#include "gblu_internal.h"

namespace gblu {

namespace {

using namespace dev;

constexpr int kThreads = kRefThreads;
constexpr int kWarps = kRefThreads / 32;
constexpr int kBatch = 4;

// ---------------------------------------------------------------------------
// slot of row r inside column k's sorted pattern, searched in [lo, hi]
// (hi clamped to the column); -1 if r is not there
__device__ __forceinline__ int find_slot(const int32_t *rows, int lo, int hi, int len, int r)
{
    if (hi > len - 1) hi = len - 1;
    if (lo > hi) return -1;
    if (rows[lo] == r) return lo;   // the lower bound is exact inside dense stretches
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (rows[mid] < r) lo = mid + 1;
        else hi = mid;
    }
    return rows[lo] == r ? lo : -1;
}

// the slots of K rows at once, each searched in its own [lo, hi] (as
// find_slot); the K bisections advance together so that their shared-memory
// loads overlap.  key < 0 marks an unused entry (slot -1).
template <int K>
__device__ __forceinline__ void find_slots(const int32_t *rows, const int (&lo0)[K], const int (&hi0)[K],
                                           int len, const int (&key)[K], int (&slot)[K])
{
    int lo[K], hi[K];
#pragma unroll
    for (int u = 0; u < K; u++) {
        lo[u] = lo0[u];
        hi[u] = min(hi0[u], len - 1);
        if (key[u] < 0 || lo[u] > hi[u]) { lo[u] = 0; hi[u] = -1; }          // nothing to search
        else if (rows[lo[u]] == key[u]) hi[u] = lo[u];                      // exact lower bound
    }
    for (;;) {
        bool more = false;
#pragma unroll
        for (int u = 0; u < K; u++) {
            if (lo[u] < hi[u]) {
                more = true;
                const int mid = (lo[u] + hi[u]) >> 1;
                if (rows[mid] < key[u]) lo[u] = mid + 1;
                else hi[u] = mid;
            }
        }
        if (!more) break;
    }
#pragma unroll
    for (int u = 0; u < K; u++) slot[u] = (lo[u] == hi[u] && rows[lo[u]] == key[u]) ? lo[u] : -1;
}

// The pivot check of step k (Algorithms 3 and 4): d = x(k), the predicted
// pivot, m = max |x| over the column's L rows (NaN if one of them is NaN).
// The threshold rule keeps the preferred row when d != 0 and |d| >= eps*m;
// a step whose preferred row went to an earlier step (strict_col) takes the
// candidate of largest magnitude, so there |d| > m.  An infinite or NaN d or
// m fails either way, and the restart reports the value.
template <typename R>
__device__ __forceinline__ bool check_pivot(const RefactorArgsT<R> &a, int k, R d, R m)
{
    if (k == a.force_col || !(d != R(0)) || !isfinite(d)) return false;
    if (a.strict_col && a.strict_col[k]) return fabs(d) > m;
    return fabs(d) >= a.eps * m;
}

// one column, one warp.  Dependencies are applied in runs of consecutive
// columns of one supernode of L, as in the group kernel below (there with
// the full description), here with runs of at most kWarpRun columns and the
// run's triangle held in registers (lane q holds row q of it).  Every 32
// dependencies the lanes check their ready flags and load their (start,
// length) in L and their supernode links; the values are then broadcast by
// shuffles.
constexpr int kWarpRun = 8;

template <typename R, bool kWait, bool kDense>
__device__ bool col_warp(const RefactorArgsT<R> &a, int k, R *xs, int32_t *rs, int lane,
                         int epoch)
{
    if (a.skip_done && ld_acquire(a.finish + k) == epoch) return false;   // final already
    const int64_t beg = __ldg(a.LUp + k);
    const int len = (int)(__ldg(a.LUp + k + 1) - beg);
    const int nU = __ldg(a.nU + k);
    // with a dense tail, a column of the block applies only its dependencies
    // before the block (its first dense_s0 rows); the block does the rest
    const bool dcol = kDense && k >= a.dense_p;
    const int nD = dcol ? __ldg(a.dense_s0 + (k - a.dense_p)) : nU - 1;
    const bool in_smem = len <= a.cap_short;
    R *x = in_smem ? xs : a.LUx + beg;
    const int32_t *rows = in_smem ? rs : a.LUi + beg;
    for (int i = lane; i < len; i += 32) {
        if (in_smem) rs[i] = __ldg(a.LUi + beg + i);
        x[i] = 0.0;
    }
    __syncwarp();
    {
        const int c = __ldg(a.Q + k);
        const int ab = __ldg(a.Ap + c), ae = __ldg(a.Ap + c + 1);
        for (int e = ab + lane; e < ae; e += 32) x[__ldg(a.amap + e)] = (R)__ldg(a.Ax + e);
    }
    __syncwarp();

    int ready = 0, mbase = 0;
    long long m_lb = 0;
    int m_nl = 0;
    unsigned cont = 0;   // bit q: dependency mbase+q continues the run of mbase+q-1
    for (int t = 0; t < nD;) {
        if (t >= ready) {
            const int tt = t + lane;
            const int jj = tt < nD ? rows[tt] : -1;
            bool ok = true;
            int ch = 0;
            if (jj >= 0) {
                // structure first: an acquire load holds back the loads after it
                m_lb = __ldg(a.LUp + jj) + __ldg(a.nU + jj);
                m_nl = (int)(__ldg(a.LUp + jj + 1) - m_lb);
                ch = __ldg(a.chain + jj);
                if (kWait) ok = ld_acquire(a.finish + jj) == epoch;
            }
            const int jp = __shfl_up_sync(kFull, jj, 1);
            const int cp = __shfl_up_sync(kFull, ch, 1);
            cont = __ballot_sync(kFull, lane > 0 && jj >= 0 && jj == jp + 1 && cp != 0);
            const unsigned m = __ballot_sync(kFull, ok);
            int run = (m == kFull) ? 32 : __ffs(~m) - 1;
            if (run == 0) {
                long long it = 0;
                while (ld_acquire(a.finish + rows[t]) != epoch) {
                    // the shared control words are read only every 32 polls
                    ++it;
                    if ((it & 31) == 0 && (ld_volatile(&a.ctl->interrupted) || ld_volatile(&a.ctl->status)))
                        return true;
                    if (it > a.spin_limit) {
                        if (lane == 0) {
                            set_status(a.ctl, GBLU_ERR_DEVICE_TIMEOUT);
                            a.ctl->where = 1;
                            a.ctl->where_k = k;
                        }
                        return true;
                    }
                    if (it > 64) __nanosleep(64);
                }
                run = 1;
            }
            ready = t + run;
            mbase = t;
            __syncwarp();
        }
        const int q0 = t - mbase;
        int w = 1;
        while (w < kWarpRun && t + w < ready && ((cont >> (q0 + w)) & 1u)) ++w;
        if (w < kWarpRun && t > mbase && t + w == mbase + 32 && t + w < nD) {
            ready = t;   // the run reaches the end of the staged window: stage from its start
            continue;
        }
        if (w > 1) {   // triangle: lane q < w holds x(j+q)
            R tv[kWarpRun - 1];
#pragma unroll
            for (int d = 0; d < kWarpRun - 1; d++) {
                const long long lbd = __shfl_sync(kFull, m_lb, (q0 + d) & 31);
                tv[d] = (d < w - 1 && lane > d && lane < w) ? __ldcg(a.LUx + lbd + (lane - d - 1)) : R(0);
            }
            R v = lane < w ? x[t + lane] : R(0);
#pragma unroll
            for (int d = 0; d < kWarpRun - 1; d++) {
                if (d < w - 1) {
                    const R mv = __shfl_sync(kFull, v, d);
                    if (lane > d && lane < w) v = fma(-tv[d], mv, v);
                }
            }
            if (lane < w) x[t + lane] = v;
            __syncwarp();
        }
        {   // rectangle: rows of R = L(:, j+w-1), multipliers x(t .. t+w-1)
            const int tl = t + w - 1;
            const int jl = rows[tl];
            const long long lbl = __shfl_sync(kFull, m_lb, q0 + w - 1);
            const int nR = __shfl_sync(kFull, m_nl, q0 + w - 1);
            bool bad = false;
            for (int r0 = 0; r0 < nR; r0 += 32 * kBatch) {
                int sl[kBatch], key[kBatch], lo[kBatch], hi[kBatch];
                R v[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; u++) {
                    const int r = r0 + u * 32 + lane;
                    key[u] = r < nR ? __ldg(a.LUi + lbl + r) : -1;
                    lo[u] = tl + 1 + r;
                    hi[u] = tl + (key[u] - jl);
                }
                find_slots<kBatch>(rows, lo, hi, len, key, sl);
#pragma unroll
                for (int u = 0; u < kBatch; u++) {
                    if (key[u] >= 0 && sl[u] < 0) bad = true;
                    v[u] = sl[u] >= 0 ? x[sl[u]] : R(0);
                }
#pragma unroll 8
                for (int d = 0; d < w; d++) {
                    const R mv = x[t + d];
                    const long long lbd = __shfl_sync(kFull, m_lb, q0 + d);
                    const R *lv = a.LUx + lbd + (w - 1 - d) + r0 + lane;
#pragma unroll
                    for (int u = 0; u < kBatch; u++)
                        if (sl[u] >= 0) v[u] = fma(-mv, __ldcg(lv + u * 32), v[u]);
                }
#pragma unroll
                for (int u = 0; u < kBatch; u++)
                    if (sl[u] >= 0) x[sl[u]] = v[u];
            }
            if (__any_sync(kFull, bad)) {  // inconsistent pattern: never index with it
                if (lane == 0) set_status(a.ctl, GBLU_ERR_INTERNAL);
                return true;
            }
        }
        __syncwarp();
        t += w;
    }

    if (dcol) {   // U above the block is final; rows >= dense_p go to the block
        R *Sc = a.S + (int64_t)(k - a.dense_p) * a.dense_ld;
        if (in_smem)
            for (int i = lane; i < nD; i += 32) a.LUx[beg + i] = xs[i];
        for (int i = nD + lane; i < len; i += 32) Sc[i - nD] = x[i];
        return false;
    }
    // m = max |x(L rows)|, NaN if one of them is NaN; with an infinite m or
    // pivot the check fails too, and the restart reports the value
    const R d = x[nU - 1];
    R m = R(0);
    for (int i = nU + lane; i < len; i += 32) m = max_nan(m, fabs(x[i]));
    m = warp_max(m);
    const bool pass = check_pivot(a, k, d, m);
    if (!pass) {
        if (lane == 0) {
            if (!a.no_stop) atomicExch(&a.ctl->interrupted, 1);
            atomicMin(&a.ctl->first_bad, k);
        }
        if (!a.no_stop) return false;
    }
    const R inv = pass ? R(1) / d : R(1);   // a failed column stays unnormalized
    if (in_smem) {
        for (int i = lane; i < len; i += 32) a.LUx[beg + i] = (i < nU) ? xs[i] : xs[i] * inv;
    } else {
        for (int i = nU + lane; i < len; i += 32) x[i] = x[i] * inv;
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(a.finish + k, epoch);
    return false;
}

// ---------------------------------------------------------------------------
// One column computed by a group of NW warps: the whole CTA, or one half of
// it for a pair of medium columns (work vector of up to cap entries in
// shared memory; longer columns are updated in place in global memory).
//
// Dependencies are applied in runs j, j+1, ..., j+w-1 (w <= 32) of
// consecutive columns of one supernode of L (chain[j+d] set for d < w-1):
// then L(:,j+d) = {j+d+1, ..., j+w-1} followed by R, the rows of L(:,j+w-1),
// so the run updates x in two parts:
//   triangle  - x(j+q) for q < w: the unit lower triangular solve of the
//               run's diagonal block (lane q of one warp holds x(j+q));
//   rectangle - every row r of R: x(r) -= L(r, j+d) * x(j+d) for d = 0..w-1,
//               one thread per row, the slot of r searched once per run.
// Every update is one fused multiply-add applied in ascending dependency
// order, exactly as when the dependencies are applied one at a time, so the
// result does not depend on how the dependencies fall into runs.
//
// The warps are specialised.  While the workers (warps 1..NW-1) apply run i
// to the rows of R whose slots lie beyond the next 32 slots, the leader
// (warp 0) applies run i to the rows in those 32 slots (they hold every row
// of run i+1), checks the ready flags of the next dependencies (staging 32
// at a time in registers, waiting if needed), solves the triangle of run
// i+1 and publishes its descriptor; one barrier per run.
constexpr int kMaxRun = 32;
constexpr int kTri = kMaxRun * (kMaxRun - 1) / 2;   // strictly lower triangle
constexpr int kRows = 2;                            // rows of R per thread per pass

// offset of column d of the staged triangle (column d holds kMaxRun-1-d rows)
__device__ __forceinline__ int tri_off(int d) { return d * (kMaxRun - 1) - d * (d - 1) / 2; }

// group barrier: the whole CTA (NW == 8) or one half (named barrier 1 + g)
template <int NW>
__device__ __forceinline__ void group_sync(int g)
{
    if (NW == kWarps) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(NW * 32) : "memory");
}

// a run as published by the leader
struct RunDesc {
    long long base[kMaxRun];   // value of R entry r for dependency d: LUx[base[d] + r]
    long long lbl;             // start of R's rows in LUi
    int t, w, jl, nR, done;
    int small;                 // nR <= kSmallRun: the leader alone applies every row
};

// a run whose rectangle has at most this many rows is applied by the leader
// warp alone (a row per lane), without waking the workers: a chain of such
// runs then costs one group barrier instead of one per run
constexpr int kSmallRun = 32;

// shared state of one group (declared once per CTA, for up to two groups)
template <typename R>
struct GroupShared {
    RunDesc run[2];            // double buffered by run parity
    R red[kWarps];
    R tri[kTri];               // the leader's staged triangle, column d at tri_off(d)
    int stop;
    int pull_slot;                 // the scratch of the wide column in progress
    unsigned long long pull_tag;   // and its tag there
};

// Wide columns (Schedule::pull_start): many dependencies in short supernode
// runs and a short L part, like the rails of a bordered matrix, on which
// every grid column depends.  The dependency loop would apply thousands of
// runs of a few columns one after another, each costing a barrier and a
// round trip through L2.  Instead the first p0 dependencies, j = rows[0..p0),
// are applied row by row through the rows of L (CSR Lrp, Lcol, Lslot), by
// the whole CTA:
//   - the prefix rows r (U entries above rows[p0]) form a sparse unit lower
//     triangular system: x(r) = A(r,k) - sum L(r,j) x(j) over row r of L in
//     ascending j, taking only j of the prefix.  One thread per row, each
//     thread's rows in ascending order, each term waiting for x(j) to be
//     published in a dense per-CTA scratch (a sentinel until then; a per-CTA
//     tag marks the prefix's entries).  The fused multiply-adds come in the
//     order of the dependency loop, so these entries are the same bits.
//   - every later row (the other U rows, the diagonal, the L rows) subtracts
//     the sum over the prefix of its row of L: one warp per row, lanes over
//     the entries, then a tree (these additions come in another order).
// The dependency loop then goes on from dependency p0.  The scratch is one of
// pull_slots, held while the prefix is computed (a CTA takes a free one;
// there are as many as CTAs fit on the device).  Returns false if a wait
// gave up (the column stops).
// the fields pull_rows reads (the instantiations without wide columns do
// not compile it in)
struct PullArgs {
    const int64_t *Lrp;
    const int32_t *Lcol, *Lslot;
    const double *LUx;
    const int32_t *finish;
    double *pull_x;
    unsigned long long *pull_tag, *pull_ctr;
    int32_t *pull_lock;
    DevCtl *ctl;
    long long spin_limit;
    int32_t pull_slots, n;
};

__device__ __forceinline__ PullArgs pull_args(const RefactorArgsT<double> &a)
{
    return PullArgs{a.Lrp,    a.Lcol,     a.Lslot,    a.LUx, a.finish,     a.pull_x,     a.pull_tag,
                    a.pull_ctr, a.pull_lock, a.ctl, a.spin_limit, a.pull_slots, a.n};
}

template <bool kWait>
__device__ __forceinline__ bool pull_rows(const PullArgs a, int k, double *x, const int32_t *rows, int len, int p0,
                                       int epoch, int tid, GroupShared<double> &sh)
{
    const int lane = tid & 31, warp = tid >> 5;
    bool fail = false;
    if (tid == 0) {
        int slot = -1;
        for (long long it = 0; slot < 0; ++it) {
            const int c = (int)((blockIdx.x + it) % a.pull_slots);
            if (atomicCAS(a.pull_lock + c, 0, 1) == 0) {
                slot = c;
            } else if (it > a.spin_limit) {
                set_status(a.ctl, GBLU_ERR_DEVICE_TIMEOUT);
                a.ctl->where = 11;
                a.ctl->where_k = k;
                break;
            }
        }
        sh.pull_slot = slot;
        if (slot >= 0) sh.pull_tag = ++a.pull_ctr[slot];
    }
    __syncthreads();
    const int slot = sh.pull_slot;
    if (slot < 0) return false;
    double *xd = a.pull_x + (size_t)slot * a.n;
    unsigned long long *xt = a.pull_tag + (size_t)slot * a.n;
    const unsigned long long tag = sh.pull_tag;
    auto release = [&]() {
        __syncthreads();
        if (tid == 0) atomicExch(a.pull_lock + slot, 0);
    };
    auto give_up = [&](long long it, int site) -> bool {
        if ((it & 31) == 0 && (ld_volatile(&a.ctl->interrupted) || ld_volatile(&a.ctl->status))) return true;
        if (it > a.spin_limit) {
            set_status(a.ctl, GBLU_ERR_DEVICE_TIMEOUT);
            a.ctl->where = site;
            a.ctl->where_k = k;
            return true;
        }
        if (it > 64) __nanosleep(64);
        return false;
    };
    // the prefix's dependencies are final
    if (kWait)
        for (int s = tid; s < p0 && !fail; s += kThreads) {
            const int j = rows[s];
            for (long long it = 1; ld_acquire(a.finish + j) != epoch; ++it)
                if (give_up(it, 9)) {
                    fail = true;
                    break;
                }
        }
    if (__syncthreads_or(fail)) {
        release();
        return false;
    }
    const double sent = __longlong_as_double((long long)kSentinel);
    for (int s = tid; s < p0; s += kThreads) {
        st_relaxed_f64(xd + rows[s], sent);
        st_relaxed_u64(xt + rows[s], tag);
    }
    __syncthreads();
    for (int s = tid; s < p0 && !fail; s += kThreads) {
        const int r = rows[s];
        double acc = x[s];
        const int64_t e1 = __ldg(a.Lrp + r + 1);
        for (int64_t e = __ldg(a.Lrp + r); e < e1; e++) {
            const int j = __ldg(a.Lcol + e);
            if (ld_relaxed_u64(xt + j) != tag) continue;
            const double l = __ldcg(a.LUx + __ldg(a.Lslot + e));
            unsigned long long b = ld_relaxed_u64(xd + j);
            for (long long it = 1; b == kSentinel; ++it) {
                if (give_up(it, 10)) {
                    fail = true;
                    break;
                }
                b = ld_relaxed_u64(xd + j);
            }
            if (fail) break;
            acc = fma(-__longlong_as_double((long long)b), l, acc);
        }
        x[s] = acc;
        st_relaxed_f64(xd + r, acc);
    }
    if (__syncthreads_or(fail)) {
        release();
        return false;
    }
    const int jlim = rows[p0 - 1];   // the last dependency of the prefix
    for (int s = p0 + warp; s < len; s += kWarps) {
        const int r = rows[s];
        const int64_t e1 = __ldg(a.Lrp + r + 1);
        double part = 0.0;
        for (int64_t e0 = __ldg(a.Lrp + r) + lane; e0 < e1; e0 += 32 * 4) {
            int j[4];
            double l[4], v[4];
            unsigned long long tg[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int64_t e = e0 + 32 * u;
                j[u] = e < e1 ? __ldg(a.Lcol + e) : INT_MAX;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const bool in = j[u] <= jlim;   // ascending: the rest is past the prefix
                tg[u] = in ? ld_relaxed_u64(xt + j[u]) : 0ull;
                l[u] = in ? __ldcg(a.LUx + __ldg(a.Lslot + e0 + 32 * u)) : 0.0;
                v[u] = in ? __longlong_as_double((long long)ld_relaxed_u64(xd + j[u])) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (j[u] <= jlim && tg[u] == tag) part = fma(v[u], l[u], part);
            if (j[3] > jlim) break;
        }
        part = warp_sum(part);
        if (lane == 0) x[s] -= part;
    }
    release();
    return true;
}

template <typename R, bool kWait, bool kDense, int NW, bool kPull>
__device__ bool col_grp(const RefactorArgsT<R> &a, int k, R *xs, int32_t *rs, int epoch, int g, int cap,
                        GroupShared<R> &sh)
{
    static_assert(NW >= 2, "a group needs a leader and workers");
    constexpr int kT = NW * 32, kTw = (NW - 1) * 32;
    if (a.skip_done && ld_acquire(a.finish + k) == epoch) return false;   // final already (uniform in the group)
    const int tid = threadIdx.x - g * kT, lane = tid & 31, warp = tid >> 5;
    const int64_t beg = __ldg(a.LUp + k);
    const int len = (int)(__ldg(a.LUp + k + 1) - beg);
    const int nU = __ldg(a.nU + k);
    // with a dense tail, a column of the block applies only its dependencies
    // before the block (its first dense_s0 rows); the block does the rest
    const bool dcol = kDense && k >= a.dense_p;
    const int nD = dcol ? __ldg(a.dense_s0 + (k - a.dense_p)) : nU - 1;
    // up to cap entries: work vector and rows in shared memory; up to as many
    // rows as the shared area holds (in double precision 3*cap for a whole
    // CTA, whose row area follows its work-vector area, and 2*cap for half a
    // CTA): the rows alone (slot searches stay in shared memory), the work
    // vector in place in global memory; longer: both in global memory
    const bool in_smem = len <= cap;
    const bool joined = reinterpret_cast<const unsigned char *>(rs) == reinterpret_cast<const unsigned char *>(xs + cap);
    const int row_cap = joined ? cap * (int)((sizeof(R) + sizeof(int32_t)) / sizeof(int32_t))
                               : cap * (int)(sizeof(R) / sizeof(int32_t));
    const bool rows_smem = !in_smem && len <= row_cap;
    int32_t *rsw = reinterpret_cast<int32_t *>(xs);   // rows over the work-vector area
    R *x = in_smem ? xs : a.LUx + beg;
    const int32_t *rows = in_smem ? rs : (rows_smem ? rsw : a.LUi + beg);
    for (int i = tid; i < len; i += kT) {
        if (in_smem) rs[i] = __ldg(a.LUi + beg + i);
        else if (rows_smem) rsw[i] = __ldg(a.LUi + beg + i);
        x[i] = 0.0;
    }
    if (tid == 0) {
        sh.stop = 0;
        sh.run[0].done = 0;
        sh.run[1].done = 0;
    }
    group_sync<NW>(g);
    {
        const int c = __ldg(a.Q + k);
        const int ab = __ldg(a.Ap + c), ae = __ldg(a.Ap + c + 1);
        for (int e = ab + tid; e < ae; e += kT) x[__ldg(a.amap + e)] = (R)__ldg(a.Ax + e);
    }
    group_sync<NW>(g);
    // a wide column: its first p0 dependencies row by row (pull_rows)
    int p0 = 0;
    if constexpr (kPull && NW == kWarps && std::is_same<R, double>::value) {
        if (a.pull_start && !dcol) p0 = min(__ldg(a.pull_start + k), nD);
        if (p0 > 0 && !pull_rows<kWait>(pull_args(a), k, x, rows, len, p0, epoch, tid, sh)) return true;
    }

    // ---- leader state: the staged window of dependencies [mbase, mbase+32),
    // lane q holding dependency mbase+q; [mbase, ready) are ready
    int ready = 0, mbase = 0;
    long long m_lb = 0;
    int m_nl = 0;
    unsigned cont = 0;   // bit q: dependency mbase+q continues the run of mbase+q-1

    // leader: find the run starting at dependency t (waiting for it to be
    // ready), solve its triangle and publish it as run[p]; false = stop
    auto lead_next = [&](int t, int p) -> bool {
        int w = 1;
        for (;;) {
            if (t >= ready) {
                const int tt = t + lane;
                const int jj = tt < nD ? rows[tt] : -1;
                bool ok = true;
                int ch = 0;
                if (jj >= 0) {
                    // structure first: an acquire load holds back the loads after it
                    m_lb = __ldg(a.LUp + jj) + __ldg(a.nU + jj);
                    m_nl = (int)(__ldg(a.LUp + jj + 1) - m_lb);
                    ch = __ldg(a.chain + jj);
                    if (kWait) ok = ld_acquire(a.finish + jj) == epoch;
                }
                const int jp = __shfl_up_sync(kFull, jj, 1);
                const int cp = __shfl_up_sync(kFull, ch, 1);
                cont = __ballot_sync(kFull, lane > 0 && jj >= 0 && jj == jp + 1 && cp != 0);
                const unsigned m = __ballot_sync(kFull, ok);
                int run = (m == kFull) ? 32 : __ffs(~m) - 1;
                if (kWait && run == 0) {
                    long long it = 0;
                    while (ld_acquire(a.finish + rows[t]) != epoch) {
                        // the shared control words are read only every 32 polls
                        ++it;
                        if ((it & 31) == 0 && (ld_volatile(&a.ctl->interrupted) || ld_volatile(&a.ctl->status)))
                            return false;
                        if (it > a.spin_limit) {
                            if (lane == 0) {
                                set_status(a.ctl, GBLU_ERR_DEVICE_TIMEOUT);
                                a.ctl->where = 1;
                                a.ctl->where_k = k;
                            }
                            return false;
                        }
                        if (it > 64) __nanosleep(64);
                    }
                    run = 1;
                }
                ready = t + run;
                mbase = t;
            }
            const int q0 = t - mbase;
            w = 1;
            while (t + w < ready && ((cont >> (q0 + w)) & 1u)) ++w;
            if (t > mbase && t + w == mbase + 32 && t + w < nD) {
                ready = t;   // the run reaches the end of the staged window: stage from its start
                continue;
            }
            break;
        }
        const int q0 = t - mbase;
        const long long lbq = __shfl_sync(kFull, m_lb, (q0 + lane) & 31);   // lane d: dependency t+d
        if (w > 1) {   // triangle: column d of the run gives its first w-1-d L entries
            for (int d0 = 0; d0 < w - 1; d0 += 8) {   // eight loads in flight
                R tv[8];
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const long long lbd = __shfl_sync(kFull, lbq, (d0 + u) & 31);
                    tv[u] = (d0 + u < w - 1 && lane < w - 1 - (d0 + u)) ? __ldcg(a.LUx + lbd + lane) : R(0);
                }
#pragma unroll
                for (int u = 0; u < 8; u++)
                    if (d0 + u < w - 1 && lane < w - 1 - (d0 + u)) sh.tri[tri_off(d0 + u) + lane] = tv[u];
            }
            __syncwarp();
            R v = lane < w ? x[t + lane] : R(0);
            for (int d = 0; d < w - 1; ++d) {
                const R mv = __shfl_sync(kFull, v, d);
                if (lane > d && lane < w) v = fma(-sh.tri[tri_off(d) + lane - d - 1], mv, v);
            }
            if (lane < w) x[t + lane] = v;
        }
        RunDesc &r = sh.run[p];
        if (lane < w) r.base[lane] = lbq + (w - 1 - lane);
        const long long lbl = __shfl_sync(kFull, lbq, w - 1);
        const int nRl = __shfl_sync(kFull, m_nl, (q0 + w - 1) & 31);
        if (lane == 0) {
            r.t = t;
            r.w = w;
            r.jl = rows[t + w - 1];
            r.lbl = lbl;
            r.nR = nRl;
            r.small = nRl <= kSmallRun;
            r.done = 0;
        }
        return true;
    };

    if (warp == 0) {
        if (p0 >= nD) {
            if (lane == 0) sh.run[0].done = 1;
        } else if (!lead_next(p0, 0) && lane == 0) {
            sh.stop = 1;
        }
    }
    group_sync<NW>(g);

    for (int i = 0;; ++i) {
        if (sh.stop == 2) {  // inconsistent pattern: never index with it
            if (tid == 0) set_status(a.ctl, GBLU_ERR_INTERNAL);
            return true;
        }
        if (sh.stop) return true;
        const RunDesc &r = sh.run[i & 1];
        if (r.done) break;
        const int t = r.t, w = r.w, nR = r.nR, jl = r.jl, small = r.small;
        const long long lbl = r.lbl;
        const int tl = t + w - 1, hend = t + w + kMaxRun;   // the leader's slots: [t+w, hend)
        bool bad = false;
        if (warp == 0) {
            // a large run: the rows of R in the leader's slots (only the first
            // 32 entries of R can fall there); a small run: every row of R, and
            // so on through the small runs that follow, while the workers wait
            // at the barrier; the run that ends the chain (or the first run
            // after a large one) is published
            const RunDesc *cur = &r;
            const bool all = small != 0;
            const int p = (i + 1) & 1;
            for (;;) {
                const int ct = cur->t, cw = cur->w, cnR = cur->nR, cjl = cur->jl;
                const long long clbl = cur->lbl;
                const int ctl = ct + cw - 1, chend = all ? INT_MAX : ct + cw + kMaxRun;
                const int nrow = all ? cnR : min(cnR, 32);
                for (int rr = lane; rr < nrow; rr += 32) {
                    const int row = __ldg(a.LUi + clbl + rr);
                    const int sl = find_slot(rows, ctl + 1 + rr, ctl + (row - cjl), len, row);
                    if (sl < 0) {
                        bad = true;
                    } else if (sl < chend) {
                        R v = x[sl];
                        for (int d0 = 0; d0 < cw; d0 += 8) {   // eight loads in flight
                            R lv[8];
#pragma unroll
                            for (int u = 0; u < 8; u++)
                                lv[u] = d0 + u < cw ? __ldcg(a.LUx + cur->base[d0 + u] + rr) : R(0);
#pragma unroll
                            for (int u = 0; u < 8; u++)
                                if (d0 + u < cw) v = fma(-x[ct + d0 + u], lv[u], v);
                        }
                        x[sl] = v;
                    }
                }
                __syncwarp();
                const int tn = ct + cw;
                if (__any_sync(kFull, bad)) break;
                if (tn >= nD) {
                    if (lane == 0) sh.run[p].done = 1;
                    break;
                }
                if (!lead_next(tn, p)) {
                    if (lane == 0) sh.stop = 1;
                    break;
                }
                __syncwarp();
                // after a large run the workers may still be updating rows of
                // the next one: a small run that follows waits for the barrier
                if (!all || !sh.run[p].small) break;
                cur = &sh.run[p];   // only the leader reads this buffer before the barrier
            }
        } else if (!small) {
            const int wt = tid - 32;
            for (int r0 = 0; r0 < nR; r0 += kRows * kTw) {
                int sl[kRows], key[kRows], lo[kRows], hi[kRows];
                R v[kRows];
#pragma unroll
                for (int u = 0; u < kRows; u++) {
                    const int rr = r0 + u * kTw + wt;
                    key[u] = rr < nR ? __ldg(a.LUi + lbl + rr) : -1;
                    lo[u] = tl + 1 + rr;
                    hi[u] = tl + (key[u] - jl);
                }
                find_slots<kRows>(rows, lo, hi, len, key, sl);
#pragma unroll
                for (int u = 0; u < kRows; u++) {
                    if (key[u] >= 0 && sl[u] < 0) bad = true;
                    if (sl[u] >= 0 && sl[u] < hend) sl[u] = -1;   // the leader's
                    v[u] = sl[u] >= 0 ? x[sl[u]] : R(0);
                }
#pragma unroll 8
                for (int d = 0; d < w; d++) {
                    const R m = x[t + d];
                    const R *lv = a.LUx + r.base[d] + r0 + wt;
#pragma unroll
                    for (int u = 0; u < kRows; u++)
                        if (sl[u] >= 0) v[u] = fma(-m, __ldcg(lv + u * kTw), v[u]);
                }
#pragma unroll
                for (int u = 0; u < kRows; u++)
                    if (sl[u] >= 0) x[sl[u]] = v[u];
            }
        }
        if (bad) sh.stop = 2;
        group_sync<NW>(g);
    }

    if (dcol) {   // U above the block is final; rows >= dense_p go to the block
        R *Sc = a.S + (int64_t)(k - a.dense_p) * a.dense_ld;
        if (in_smem)
            for (int i = tid; i < nD; i += kT) a.LUx[beg + i] = xs[i];
        for (int i = nD + tid; i < len; i += kT) Sc[i - nD] = x[i];
        return false;
    }
    // m = max |x(L rows)|, NaN if one of them is NaN; with an infinite m or
    // pivot the check fails too, and the restart reports the value
    const R d = x[nU - 1];
    R m = R(0);
    for (int i = nU + tid; i < len; i += kT) m = max_nan(m, fabs(x[i]));
    m = warp_max(m);
    if (lane == 0) sh.red[warp] = m;
    group_sync<NW>(g);
    m = sh.red[0];
    for (int w = 1; w < NW; w++) m = max_nan(m, sh.red[w]);
    const bool pass = check_pivot(a, k, d, m);
    if (!pass) {
        if (tid == 0) {
            if (!a.no_stop) atomicExch(&a.ctl->interrupted, 1);
            atomicMin(&a.ctl->first_bad, k);
        }
        if (!a.no_stop) return false;
    }
    const R inv = pass ? R(1) / d : R(1);   // a failed column stays unnormalized
    if (in_smem) {
        for (int i = tid; i < len; i += kT) a.LUx[beg + i] = (i < nU) ? xs[i] : xs[i] * inv;
    } else {
        for (int i = nU + tid; i < len; i += kT) x[i] = x[i] * inv;
    }
    __threadfence();
    group_sync<NW>(g);
    if (tid == 0) st_release(a.finish + k, epoch);
    return false;
}

__global__ void begin_refactor_kernel(DevCtl *ctl)
{
    ctl->ticket = 0;
    ctl->interrupted = 0;
    ctl->first_bad = INT_MAX;
    ctl->status = 0;
    ctl->where = 0;
    ctl->where_k = -1;
}

// One task of the schedule: one long column (whole CTA), two medium
// columns (a half each) or up to 8 short ones (a warp each); true = stop.
template <typename R, bool kWait, bool kDense, bool kPull>
__device__ __forceinline__ bool run_task(const RefactorArgsT<R> &a, int tt, R *xs, int32_t *rs, int epoch,
                                         GroupShared<R> *s_grp)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = __ldg(a.task_ptr + tt), c1 = __ldg(a.task_ptr + tt + 1);
    const int k0 = __ldg(a.task_cols + c0);
    const int64_t len0 = __ldg(a.LUp + k0 + 1) - __ldg(a.LUp + k0);
    if (c1 - c0 == 1 && len0 > a.cap_short)            // one long column: whole CTA
        return col_grp<R, kWait, kDense, kWarps, kPull>(a, k0, xs, rs, epoch, 0, a.cap_long, s_grp[0]);
    if (c1 - c0 == 2 && len0 > a.cap_short) {          // two medium columns: a half each
        const int g = warp / (kWarps / 2);
        const int half = a.cap_long / 2;
        const bool hs = col_grp<R, kWait, kDense, kWarps / 2, false>(a, __ldg(a.task_cols + c0 + g), xs + (size_t)g * half,
                                                          rs + (size_t)g * half, epoch, g, half, s_grp[g]);
        return __syncthreads_or(hs);
    }
    bool ws = false;
    if (c0 + warp < c1)
        ws = col_warp<R, kWait, kDense>(a, __ldg(a.task_cols + c0 + warp), xs + (size_t)warp * a.cap_short,
                                     rs + (size_t)warp * a.cap_short, lane, epoch);
    return __syncthreads_or(ws);
}

// Tasks [task_begin, task_begin + ntasks): one per CTA in cluster mode
// (persistent == 0), taken by ticket in pipeline mode (persistent == 1).
template <typename R, bool kWait, bool kDense, bool kPull>
__global__ void __launch_bounds__(kThreads, 3) refactor_task_kernel(RefactorArgsT<R> a, int epoch, int persistent)
{
    // a replayed graph passes -1: the epoch was written to the control block
    if (epoch < 0) epoch = ld_volatile(&a.ctl->epoch);
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_t, s_quit;
    __shared__ GroupShared<R> s_grp[2];
    R *xs = reinterpret_cast<R *>(smem);
    int32_t *rs = reinterpret_cast<int32_t *>(smem + (size_t)a.cap_long * sizeof(R));
    for (int iter = 0;; ++iter) {
        if (threadIdx.x == 0) {
            s_t = persistent ? atomicAdd(&a.ctl->ticket, 1) : (iter == 0 ? (int)blockIdx.x : a.ntasks);
            s_quit = ld_volatile(&a.ctl->interrupted) || ld_volatile(&a.ctl->status);
        }
        __syncthreads();
        const int t = s_t, quit = s_quit;
        __syncthreads();
        if (t >= a.ntasks || quit) break;
        if (run_task<R, kWait, kDense, kPull>(a, a.task_begin + t, xs, rs, epoch, s_grp)) break;
    }
}

// Batch of value sets on one structure: sets[s] is the argument block of
// set s (its A values, factor values, ready flags and control block; the
// structure fields are shared).  The sets go in groups of `group`: the
// tickets of a group are its tasks in order, each for all the group's sets
// (task-major inside the group), and the next group follows; so every set
// meets its tasks in a topological order, and only a group's factors are
// being read at a time.  A set whose check failed (or whose wait gave up)
// is skipped from then on; the other sets go on.
// ticket t of a batch in groups of g sets (the last group may be smaller):
// the group's tickets are task-major, set-minor
__device__ __forceinline__ void group_split(long long t, int ntasks, int nsets, int g, int &task, int &set)
{
    const long long full = (long long)(nsets / g) * g;   // sets in full groups
    const long long tf = (long long)ntasks * full;
    if (t < tf) {
        const long long gi = t / ((long long)ntasks * g), r = t % ((long long)ntasks * g);
        task = (int)(r / g);
        set = (int)(gi * g + r % g);
    } else {
        const long long r = t - tf, gl = nsets - full;
        task = (int)(r / gl);
        set = (int)(full + r % gl);
    }
}
__device__ __forceinline__ int group_set(long long t, int ntasks, int nsets, int g)
{
    int task, set;
    group_split(t, ntasks, nsets, g, task, set);
    return set;
}
__device__ __forceinline__ int group_task(long long t, int ntasks, int nsets, int g)
{
    int task, set;
    group_split(t, ntasks, nsets, g, task, set);
    return task;
}

template <bool kWait, bool kPull>
__global__ void __launch_bounds__(kThreads, 3)
refactor_batch_kernel(const RefactorArgs *sets, int nsets, int task_begin, int ntasks, int epoch, int persistent,
                      int32_t *ticket, const SetTask *order, int group)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_t, s_skip;
    __shared__ GroupShared<double> s_grp[2];
    double *xs = reinterpret_cast<double *>(smem);
    int32_t *rs = reinterpret_cast<int32_t *>(smem + (size_t)sets[0].cap_long * sizeof(double));
    // ticket t: task t / nsets of set t % nsets, or, with an order array
    // (sets of different patterns), the (set, task) pair order[t]
    const long long total = order ? (long long)ntasks : (long long)ntasks * nsets;
    for (int iter = 0;; ++iter) {
        if (threadIdx.x == 0) {
            const long long t = persistent ? (long long)atomicAdd(ticket, 1) : (iter == 0 ? (long long)blockIdx.x : total);
            s_t = t < total ? (int)t : -1;
            s_skip = 0;
            if (t < total) {
                const int si = order ? __ldg(&order[t].set) : group_set(t, ntasks, nsets, group);
                const DevCtl *c = sets[si].ctl;
                s_skip = ld_volatile(&c->interrupted) || ld_volatile(&c->status);
            }
        }
        __syncthreads();
        const int t = s_t, skip = s_skip;
        __syncthreads();
        if (t < 0) break;
        if (skip) continue;
        const int si = order ? __ldg(&order[t].set) : group_set(t, ntasks, nsets, group);
        const int task = order ? __ldg(&order[t].task) : task_begin + group_task(t, ntasks, nsets, group);
        // a local copy: stores through the work vector cannot alias it, so its
        // fields stay in registers instead of being reloaded from memory
        const RefactorArgs as = sets[si];
        run_task<double, kWait, false, kPull>(as, task, xs, rs, epoch, s_grp);
    }
}

// control blocks of sets that each have their own (multi-pattern batches)
__global__ void begin_multi_kernel(const RefactorArgs *sets, int nsets, int32_t *ticket)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsets; s += gridDim.x * blockDim.x) {
        DevCtl *c = sets[s].ctl;
        c->ticket = 0;
        c->interrupted = 0;
        c->first_bad = INT_MAX;
        c->status = 0;
        c->where = 0;
        c->where_k = -1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *ticket = 0;
}

__global__ void begin_batch_kernel(DevCtl *ctl, int nsets, int32_t *ticket)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsets; s += gridDim.x * blockDim.x) {
        ctl[s].ticket = 0;
        ctl[s].interrupted = 0;
        ctl[s].first_bad = INT_MAX;
        ctl[s].status = 0;
        ctl[s].where = 0;
        ctl[s].where_k = -1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *ticket = 0;
}

template <typename R>
size_t task_smem(const RefactorArgsT<R> &a)
{
    return (size_t)a.cap_long * (sizeof(R) + sizeof(int32_t));
}

}  // namespace

int launch_begin_refactor(DevCtl *ctl, void *stream)
{
    begin_refactor_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(ctl);
    return (int)cudaGetLastError();
}

// the shared-memory allowance of every instantiation of a kernel template
template <class K>
static cudaError_t allow_smem(K kernel, size_t sm, cudaError_t e)
{
    return e == cudaSuccess ? cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) : e;
}

int refactor_setup(int cap_long, int *blocks_per_sm, int *batch_blocks_per_sm)
{
    const size_t sm = (size_t)cap_long * (sizeof(double) + sizeof(int32_t));
    cudaError_t e = cudaSuccess;
    e = allow_smem(refactor_task_kernel<double, true, false, false>, sm, e);
    e = allow_smem(refactor_task_kernel<double, false, false, false>, sm, e);
    e = allow_smem(refactor_task_kernel<double, true, true, false>, sm, e);
    e = allow_smem(refactor_task_kernel<double, false, true, false>, sm, e);
    e = allow_smem(refactor_task_kernel<double, true, false, true>, sm, e);
    e = allow_smem(refactor_task_kernel<double, false, false, true>, sm, e);
    e = allow_smem(refactor_batch_kernel<true, false>, sm, e);
    e = allow_smem(refactor_batch_kernel<false, false>, sm, e);
    e = allow_smem(refactor_batch_kernel<true, true>, sm, e);
    e = allow_smem(refactor_batch_kernel<false, true>, sm, e);
    if (e != cudaSuccess) return (int)e;
    // persistent grids are sized for the instantiation that fits fewest
    int b[3] = {0, 0, 0};
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[0], refactor_task_kernel<double, true, false, false>, kThreads, sm);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[1], refactor_task_kernel<double, true, true, false>, kThreads, sm);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[2], refactor_task_kernel<double, true, false, true>, kThreads, sm);
    *blocks_per_sm = std::min(b[0], std::min(b[1], b[2]));
    // the batch kernel keeps a copy of its set's argument block (it spills a
    // few registers at three CTAs per SM, which measured faster than two)
    int c[2] = {0, 0};
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c[0], refactor_batch_kernel<true, false>, kThreads, sm);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c[1], refactor_batch_kernel<true, true>, kThreads, sm);
    *batch_blocks_per_sm = std::min(c[0], c[1]);
    return (int)e;
}

int launch_begin_batch(DevCtl *ctl, int nsets, int32_t *ticket, void *stream)
{
    const int g = (nsets + 255) / 256;
    begin_batch_kernel<<<g < 1 ? 1 : g, 256, 0, (cudaStream_t)stream>>>(ctl, nsets, ticket);
    return (int)cudaGetLastError();
}

int launch_refactor_batch(const RefactorArgs *sets_dev, const RefactorArgs &a0, int nsets, bool pipeline,
                          int grid, int epoch, int32_t *ticket, void *stream, int group)
{
    if (a0.ntasks <= 0 || nsets <= 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (group < 1 || group > nsets) group = nsets;
    if (pipeline) {
        if (a0.pull_start)
            refactor_batch_kernel<true, true><<<grid, kThreads, task_smem(a0), st>>>(
                sets_dev, nsets, a0.task_begin, a0.ntasks, epoch, 1, ticket, nullptr, group);
        else
            refactor_batch_kernel<true, false><<<grid, kThreads, task_smem(a0), st>>>(
                sets_dev, nsets, a0.task_begin, a0.ntasks, epoch, 1, ticket, nullptr, group);
    } else {
        // a level launch has no waits: one group holding every set
        const long long blocks = (long long)a0.ntasks * nsets;
        if (blocks > INT_MAX) return (int)cudaErrorInvalidValue;
        if (a0.pull_start)
            refactor_batch_kernel<false, true><<<(unsigned)blocks, kThreads, task_smem(a0), st>>>(
                sets_dev, nsets, a0.task_begin, a0.ntasks, epoch, 0, ticket, nullptr, nsets);
        else
            refactor_batch_kernel<false, false><<<(unsigned)blocks, kThreads, task_smem(a0), st>>>(
                sets_dev, nsets, a0.task_begin, a0.ntasks, epoch, 0, ticket, nullptr, nsets);
    }
    return (int)cudaGetLastError();
}

int launch_refactor_multi(const RefactorArgs *sets_dev, const RefactorArgs &a0, int nsets, const SetTask *order_dev,
                          int npairs, int grid, int epoch, int32_t *ticket, void *stream, bool pull)
{
    if (npairs <= 0 || nsets <= 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    int g = (nsets + 255) / 256;
    begin_multi_kernel<<<g, 256, 0, st>>>(sets_dev, nsets, ticket);
    // pull: some set has wide columns (each set's argument block says which)
    if (pull)
        refactor_batch_kernel<true, true><<<grid, kThreads, task_smem(a0), st>>>(sets_dev, nsets, 0, npairs, epoch, 1, ticket,
                                                                       order_dev, 1);
    else
        refactor_batch_kernel<true, false><<<grid, kThreads, task_smem(a0), st>>>(sets_dev, nsets, 0, npairs, epoch, 1, ticket,
                                                                       order_dev, 1);
    return (int)cudaGetLastError();
}

int refactor_setup_f32(int cap_long, int *blocks_per_sm)
{
    const size_t sm = (size_t)cap_long * (sizeof(float) + sizeof(int32_t));
    cudaError_t e = cudaFuncSetAttribute(refactor_task_kernel<float, true, false, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(refactor_task_kernel<float, false, false, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, refactor_task_kernel<float, true, false, false>,
                                                              kThreads, sm);
}

int launch_refactor_tasks_f32(const RefactorArgsT<float> &a, bool pipeline, int grid, int epoch, void *stream)
{
    if (a.ntasks <= 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (pipeline) refactor_task_kernel<float, true, false, false><<<grid, kThreads, task_smem(a), st>>>(a, epoch, 1);
    else refactor_task_kernel<float, false, false, false><<<a.ntasks, kThreads, task_smem(a), st>>>(a, epoch, 0);
    return (int)cudaGetLastError();
}

int launch_refactor_tasks(const RefactorArgs &a, bool pipeline, int grid, int epoch, void *stream)
{
    if (a.ntasks <= 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    const bool dense = a.dense_p < INT_MAX;   // a dense tail is in use
    if (pipeline) {
        if (dense) refactor_task_kernel<double, true, true, false><<<grid, kThreads, task_smem(a), st>>>(a, epoch, 1);
        else if (a.pull_start) refactor_task_kernel<double, true, false, true><<<grid, kThreads, task_smem(a), st>>>(a, epoch, 1);
        else refactor_task_kernel<double, true, false, false><<<grid, kThreads, task_smem(a), st>>>(a, epoch, 1);
    } else {
        if (dense) refactor_task_kernel<double, false, true, false><<<a.ntasks, kThreads, task_smem(a), st>>>(a, epoch, 0);
        else if (a.pull_start)
            refactor_task_kernel<double, false, false, true><<<a.ntasks, kThreads, task_smem(a), st>>>(a, epoch, 0);
        else refactor_task_kernel<double, false, false, false><<<a.ntasks, kThreads, task_smem(a), st>>>(a, epoch, 0);
    }
    return (int)cudaGetLastError();
}

}  // namespace gblu
