// Device kernels of the sparse LU path (sm_103a).
//
//  (the checked re-factorization kernels are in refactor.cu)
//  * tail_kernel     factorization with threshold pivoting of a set of
//                    columns (Section IV-D, Algorithm 5 and Algorithm 1):
//                    one CTA per column, columns taken in increasing order
//                    by an atomic ticket, waiting on ready flags of earlier
//                    columns.
//  * lsolve/usolve   triangular solves (Algorithm 2, Section V): one warp
//                    per row on row-wise copies, level launches or values
//                    published with a NaN sentinel (sync-free).
//  * residual        ||b - A x||_inf / (||A||_inf ||x||_inf) in float64.
//
// Every wait is bounded by spin_limit iterations; on expiry the kernel
// records GBLU_ERR_DEVICE_TIMEOUT in the control block and returns.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "device_util.cuh"
#include "gblu_internal.h"

namespace gblu {

namespace {

using namespace dev;

// ---------------------------------------------------------------------------
// Factorization with threshold pivoting of the columns in a.seq (ascending),
// one CTA per column, columns handed out by an atomic ticket.
//
// Column k: scatter A(:,Q[k]) into a dense work vector x (original row ids)
// with a stamp array for the structure; then sweep the earlier steps j of
// k's column-elimination subtree range [clo[k], k) in increasing order.
// Step j is a dependency iff its pivot row is already in the structure;
// applying it, x(rows of L(:,j)) -= x(piv[j]) * L(:,j), may add rows and so
// create later dependencies, which the ascending sweep meets afterwards.  A
// step that is not finished yet is waited for (its pivot decides whether it
// is a dependency).  Then threshold pivoting with the preferred row, exactly
// as the oracle defines it, and the column is appended to the pool.
__device__ bool tail_column(const TailArgs &a, int k, double *x, int32_t *mark,
                            int32_t *list, int32_t *cls, unsigned *bm, int epoch)
{
    __shared__ int s_cnt, s_found, s_mode, s_stop;
    __shared__ double r_m[kTailThreads / 32], r_ba[kTailThreads / 32];
    __shared__ int r_bq[kTailThreads / 32], r_br[kTailThreads / 32];
    __shared__ int r_nu[kTailThreads / 32], r_nc[kTailThreads / 32], r_pc[kTailThreads / 32];
    __shared__ int s_piv, s_nu, s_nc;
    __shared__ unsigned long long s_off;
    __shared__ int s_u, s_l;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int stamp = k + 1;
    if (tid == 0) { s_cnt = 0; s_stop = 0; }
    __syncthreads();
    {
        const int c = __ldg(a.Q + k);
        for (int e = __ldg(a.Ap + c) + tid; e < __ldg(a.Ap + c + 1); e += kTailThreads) {
            const int r = __ldg(a.Ai + e);
            x[r] = __ldg(a.Ax + e);
            mark[r] = stamp;
            list[atomicAdd(&s_cnt, 1)] = r;
        }
    }
    __syncthreads();
    // x(rows of L(:,jd)) -= x(piv[jd]) * L(:,jd); rows new to the structure
    // whose step is final and below `fk` are entered in the step bitmap
    auto apply_dep = [&](int jd, int fk) {
        const int pr = __ldcg(a.piv + jd);
        const double xj = x[pr];
        const int64_t b = __ldcg(a.cbeg + jd) + __ldcg(a.cnu + jd);
        const int64_t e_end = b + __ldcg(a.cnl + jd);
        for (int64_t e = b + tid; e < e_end; e += kTailThreads) {
            const int r = __ldcg(a.rows + e);
            const double v = __ldcg(a.vals + e);
            if (mark[r] != stamp) {
                mark[r] = stamp;
                x[r] = 0.0;
                list[atomicAdd(&s_cnt, 1)] = r;
                int sr = __ldcg(a.pinv + r);
                if (sr < 0 && a.speculate) sr = __ldg(a.prefer_inv + r);
                if (sr > jd && sr < fk) atomicOr(bm + (sr >> 5), 1u << (sr & 31));
            }
            x[r] = fma(-xj, v, x[r]);
        }
    };
    int j = __ldg(a.clo + k);
    if (a.speculate) {
        // every dependency is the step of a row in the structure: the row's
        // pivot step once that step is final, else the step that pivoted it
        // before (the speculation).  One ascending walk over a step bitmap;
        // a predicted dependency that is not final yet is waited for.
        for (int i = tid; i < s_cnt; i += kTailThreads) {
            const int r = list[i];
            int sr = __ldcg(a.pinv + r);
            if (sr < 0) sr = __ldg(a.prefer_inv + r);
            if (sr >= j && sr < k) atomicOr(bm + (sr >> 5), 1u << (sr & 31));
        }
        __syncthreads();
        int cur = j;
        for (;;) {
            if (warp == 0) {
                int found = k;
                for (int wb = cur >> 5; wb * 32 < k; wb += 32) {
                    const int w = wb + lane;
                    unsigned v = w * 32 < k ? *(const volatile unsigned *)(bm + w) : 0u;
                    if (w == (cur >> 5)) v &= ~0u << (cur & 31);
                    const unsigned nz = __ballot_sync(kFull, v != 0u);
                    if (nz) {
                        const int l = __ffs(nz) - 1;
                        const unsigned vv = __shfl_sync(kFull, v, l);
                        found = min((wb + l) * 32 + __ffs(vv) - 1, k);
                        break;
                    }
                }
                if (lane == 0) {
                    s_found = found;
                    if (found < k) atomicAnd(bm + (found >> 5), ~(1u << (found & 31)));
                }
            }
            __syncthreads();
            const int jd = s_found;
            if (jd >= k) break;
            if (tid == 0) {
                long long it = 0;
                while (ld_acquire(a.done + jd) != epoch) {
                    ++it;
                    if ((it & 63) == 0 && (ld_volatile(&a.ctl->abort_tail) || ld_volatile(&a.ctl->status))) {
                        s_stop = 1;
                        break;
                    }
                    if (it > a.spin_limit) {
                        set_status(a.ctl, GBLU_ERR_DEVICE_TIMEOUT);
                        a.ctl->where = 3;
                        a.ctl->where_k = k;
                        atomicExch(&a.ctl->abort_tail, 1);
                        s_stop = 1;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __syncthreads();
            if (s_stop) {
                // leave the bitmap clean for the CTA's next column
                for (int w = (jd >> 5) + tid; w * 32 < k; w += kTailThreads) bm[w] = 0u;
                return true;
            }
            if (mark[__ldcg(a.piv + jd)] == stamp) apply_dep(jd, k);
            __syncthreads();
            cur = jd + 1;
        }
        j = k;
    }
    // ---- steps below the done frontier: every such step is final, so the
    // dependencies among them are the steps of the rows in the structure
    // (row -> step map), taken in ascending order from a bitmap
    if (warp == 0 && !a.speculate) {
        int f = ld_acquire(&a.ctl->tail_frontier);
        for (long long it = 0; f < k && it < a.n; it++) {
            const int jj = f + lane;
            const bool ok = jj < a.n && ld_acquire(a.done + jj) == epoch;
            const unsigned bb = __ballot_sync(kFull, ok);
            if (bb == kFull) {
                f += 32;
                continue;
            }
            f += __ffs(~bb) - 1;
            break;
        }
        if (lane == 0) {
            __threadfence();
            atomicMax(&a.ctl->tail_frontier, f);
            s_found = f;
        }
    }
    __syncthreads();
    const int fk = min(s_found, k);
    if (fk > j && !a.speculate) {
        for (int i = tid; i < s_cnt; i += kTailThreads) {
            const int sr = __ldcg(a.pinv + list[i]);
            if (sr >= j && sr < fk) atomicOr(bm + (sr >> 5), 1u << (sr & 31));
        }
        __syncthreads();
        int cur = j;
        for (;;) {
            if (warp == 0) {
                int found = fk;
                for (int wb = cur >> 5; wb * 32 < fk; wb += 32) {
                    const int w = wb + lane;
                    unsigned v = w * 32 < fk ? *(const volatile unsigned *)(bm + w) : 0u;
                    if (w == (cur >> 5)) v &= ~0u << (cur & 31);
                    const unsigned nz = __ballot_sync(kFull, v != 0u);
                    if (nz) {
                        const int l = __ffs(nz) - 1;
                        const unsigned vv = __shfl_sync(kFull, v, l);
                        found = min((wb + l) * 32 + __ffs(vv) - 1, fk);
                        break;
                    }
                }
                if (lane == 0) {
                    s_found = found;
                    if (found < fk) atomicAnd(bm + (found >> 5), ~(1u << (found & 31)));
                }
            }
            __syncthreads();
            const int jd = s_found;
            if (jd >= fk) break;
            apply_dep(jd, fk);
            __syncthreads();
            cur = jd + 1;
        }
        j = fk;
    }
    // ---- steps at or above the frontier, in increasing order: wait for an
    // unfinished one (its pivot decides whether it is a dependency)
    while (j < k) {
        if (warp == 0) {
            int found = k, mode = 0;
            for (int base = j; base < k; base += 32) {
                const int jj = base + lane;
                bool notready = false, dep = false;
                if (jj < k) {
                    if (ld_acquire(a.done + jj) != epoch)
                        // speculative: an unfinished step matters only if its
                        // preferred row is already in the structure (a step
                        // that takes another row is caught by tail_mispredict)
                        notready = !a.speculate || mark[__ldg(a.prefer + jj)] == stamp;
                    else
                        dep = mark[__ldcg(a.piv + jj)] == stamp;
                }
                const unsigned nr = __ballot_sync(kFull, notready);
                const unsigned dp = __ballot_sync(kFull, dep);
                const unsigned any = nr | dp;
                if (any) {
                    const int l = __ffs(any) - 1;
                    found = base + l;
                    mode = ((nr >> l) & 1u) ? 2 : 1;
                    break;
                }
            }
            if (lane == 0) { s_found = found; s_mode = mode; }
        }
        __syncthreads();
        const int found = s_found, mode = s_mode;
        if (found >= k) break;
        if (mode == 2) {
            if (tid == 0) {
                long long it = 0;
                while (ld_acquire(a.done + found) != epoch) {
                    ++it;
                    if ((it & 63) == 0 && (ld_volatile(&a.ctl->abort_tail) || ld_volatile(&a.ctl->status))) {
                        s_stop = 1;
                        break;
                    }
                    if (it > a.spin_limit) {
                        set_status(a.ctl, GBLU_ERR_DEVICE_TIMEOUT);
                        a.ctl->where = 2;
                        a.ctl->where_k = k;
                        atomicExch(&a.ctl->abort_tail, 1);
                        s_stop = 1;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __syncthreads();
            if (s_stop) return true;
            j = found;
            continue;
        }
        apply_dep(found, 0);
        __syncthreads();
        j = found + 1;
    }

    // ---- threshold pivoting (Algorithm 5 lines 14-15, preferred row) ----
    // Every row is classified once (pivotal at step cls[i] >= 0, or a
    // candidate); counting and storing both use that classification.  A
    // pivotal row must belong to a step of k's elimination subtree.
    const int cnt = s_cnt;
    const int pref = __ldg(a.prefer + k);
    const int lo_k = __ldg(a.clo + k);
    double m = 0.0, ba = 0.0;
    int bq = INT_MAX, br = -1, nu = 0, nc = 0, pc = 0, badrow = 0;
    for (int i = tid; i < cnt; i += kTailThreads) {
        const int r = list[i];
        if (!isfinite(x[r])) badrow |= 4;   // a NaN or infinite value in the column
        int pj = __ldcg(a.pinv + r);
        if (pj >= k) {
            // pivotal at a later step, which can only finish first when it
            // skipped this one speculatively: at step k the row is still a
            // candidate.  Without speculation it breaks the elimination-tree
            // bound.
            if (a.speculate) pj = -1;
            else badrow = 1;
        }
        cls[i] = pj;
        if (pj >= 0) {
            if (pj < lo_k) badrow = 1;
            nu++;
            continue;
        }
        nc++;
        const double av = fabs(x[r]);
        if (r == pref) pc = 1;
        else m = fmax(m, av);
        const int q = __ldg(a.qinv + r);
        if (av > 0.0 && (br < 0 || av > ba || (av == ba && q < bq))) { ba = av; bq = q; br = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(kFull, m, o));
        const double oa = __shfl_xor_sync(kFull, ba, o);
        const int oq = __shfl_xor_sync(kFull, bq, o), orr = __shfl_xor_sync(kFull, br, o);
        if (orr >= 0 && (br < 0 || oa > ba || (oa == ba && oq < bq))) { ba = oa; bq = oq; br = orr; }
        nu += __shfl_xor_sync(kFull, nu, o);
        nc += __shfl_xor_sync(kFull, nc, o);
        pc |= __shfl_xor_sync(kFull, pc, o);
        badrow |= __shfl_xor_sync(kFull, badrow, o);
    }
    if (lane == 0) { r_m[warp] = m; r_ba[warp] = ba; r_bq[warp] = bq; r_br[warp] = br; r_nu[warp] = nu; r_nc[warp] = nc; r_pc[warp] = pc | (badrow << 1); }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kTailThreads / 32; w++) {
            m = fmax(m, r_m[w]);
            if (r_br[w] >= 0 && (br < 0 || r_ba[w] > ba || (r_ba[w] == ba && r_bq[w] < bq))) {
                ba = r_ba[w]; bq = r_bq[w]; br = r_br[w];
            }
            nu += r_nu[w];
            nc += r_nc[w];
            pc |= r_pc[w];
        }
        badrow = (pc >> 1) | badrow;
        pc &= 1;
        const bool nonfinite = (badrow & 4) != 0;
        badrow &= 3;
        int piv = -1;
        if (pc) {
            const double xp = x[pref];
            if (xp != 0.0 && fabs(xp) >= a.eps * m) piv = pref;
        }
        if (piv < 0) piv = br;
        if (a.speculate && piv >= 0 && piv != pref) atomicMin(&a.ctl->tail_mispredict, k);
        s_stop = 0;
        if (a.speculate && (badrow || piv < 0 || nonfinite)) {
            // in a speculative pass only a wrong speculation upstream gives a
            // structure outside the elimination-tree bound or no nonzero
            // candidate: stop the pass; it is repeated from this step on
            atomicMin(&a.ctl->tail_mispredict, k - 1);
            atomicExch(&a.ctl->abort_tail, 1);
            s_stop = 1;
        } else if (nonfinite) {
            set_status(a.ctl, GBLU_ERR_NONFINITE);
            a.ctl->where_k = k;
            atomicExch(&a.ctl->abort_tail, 1);
            s_stop = 1;
        } else if (badrow) {
            set_status(a.ctl, GBLU_ERR_INTERNAL);
            a.ctl->where_k = k;
            atomicExch(&a.ctl->abort_tail, 1);
            s_stop = 1;
        } else if (piv < 0) {
            set_status(a.ctl, GBLU_ERR_SINGULAR);
            a.ctl->where_k = k;
            atomicExch(&a.ctl->abort_tail, 1);
            s_stop = 1;
        } else {
            const unsigned long long total = (unsigned long long)nu + (unsigned long long)nc;
            const unsigned long long off = atomicAdd(&a.ctl->pool_top, total);
            if (off + total > a.pool_end) {
                set_status(a.ctl, GBLU_INTERNAL_POOL_FULL);
                atomicExch(&a.ctl->abort_tail, 1);
                s_stop = 1;
            }
            s_off = off;
        }
        s_piv = piv;
        s_nu = nu;
        s_nc = nc;
        s_u = 0;
        s_l = 0;
    }
    __syncthreads();
    if (s_stop) return true;
    const int piv = s_piv;
    const unsigned long long off = s_off;
    const int nuc = s_nu;
    const double d = x[piv];
    for (int i = tid; i < cnt; i += kTailThreads) {
        const int r = list[i];
        const int pj = cls[i];
        if (pj >= 0) {
            const int p = atomicAdd(&s_u, 1);
            a.rows[off + p] = pj;
            a.vals[off + p] = x[r];
        } else if (r != piv) {
            const int p = atomicAdd(&s_l, 1);
            a.rows[off + nuc + 1 + p] = r;
            a.vals[off + nuc + 1 + p] = x[r] / d;
        }
    }
    if (tid == 0) {
        a.rows[off + nuc] = k;
        a.vals[off + nuc] = d;
        a.cbeg[k] = (int64_t)off;
        a.cnu[k] = nuc + 1;
        a.cnl[k] = s_nc - 1;
        a.pinv[piv] = k;
        a.piv[k] = piv;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release(a.done + k, epoch);
    return false;
}

__global__ void begin_tail_kernel(DevCtl *ctl, unsigned long long pool_base)
{
    ctl->tail_ticket = 0;
    ctl->tail_frontier = 0;
    ctl->tail_mispredict = INT_MAX;
    ctl->abort_tail = 0;
    ctl->status = 0;
    ctl->pool_top = pool_base;
    ctl->where = 0;
    ctl->where_k = -1;
}

__global__ void tail_init_kernel(int32_t n, const int32_t *restart, const int32_t *piv_old,
                                 int32_t *pinv, int32_t *piv, int32_t *done, int epoch)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const bool rs = restart[k] != 0;
        pinv[piv_old[k]] = rs ? -1 : k;
        piv[k] = rs ? -1 : piv_old[k];
        done[k] = rs ? 0 : epoch;
    }
}

__global__ void __launch_bounds__(kTailThreads) tail_kernel(TailArgs a, int epoch)
{
    extern __shared__ unsigned s_bits[];
    __shared__ int s_t, s_quit;
    double *x = a.sx + (size_t)blockIdx.x * a.n;
    int32_t *mark = a.smark + (size_t)blockIdx.x * a.n;
    int32_t *list = a.slist + (size_t)blockIdx.x * a.n;
    int32_t *cls = a.sclass + (size_t)blockIdx.x * a.n;
    const int words = (a.n + 31) >> 5;
    unsigned *bm = a.bits_in_smem ? s_bits : a.sbits + (size_t)blockIdx.x * words;
    if (a.bits_in_smem)   // the global bitmap is cleared by the host
        for (int w = threadIdx.x; w < words; w += kTailThreads) s_bits[w] = 0u;
    for (;;) {
        if (threadIdx.x == 0) {
            s_t = atomicAdd(&a.ctl->tail_ticket, 1);
            s_quit = ld_volatile(&a.ctl->abort_tail) || ld_volatile(&a.ctl->status);
        }
        __syncthreads();
        const int t = s_t, quit = s_quit;
        __syncthreads();
        if (t >= a.nseq || quit) break;
        if (tail_column(a, __ldg(a.seq + t), x, mark, list, cls, bm, epoch)) break;
    }
}

// ---------------------------------------------------------------------------
// Triangular solves on row-wise copies (Algorithm 2): one warp per row; the
// lanes split the row and the dot product is reduced in a fixed tree, so the
// result does not depend on the schedule.
//
// Readiness travels with the values: before each solve y (forward result)
// and z (backward result) are filled with a NaN sentinel; a row publishes its
// value with one 64-bit store, and a consumer polls the value itself with
// relaxed 64-bit loads until it is no longer the sentinel.  No flag array
// and no fence per dependency; a lane consumes each dependency as soon as it
// lands.  Backward rows walk their entries from the highest column down,
// the order in which those values are produced.

__global__ void begin_solve_kernel(DevCtl *ctl, double *y, double *z, double *el, double *eu, int n)
{
    const double sent = __longlong_as_double((long long)kSentinel);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        y[i] = sent;
        z[i] = sent;
        el[i] = sent;
        eu[i] = sent;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->ticket_l = 0;
        ctl->ticket_u = 0;
        ctl->ticket_tl = 0;
        ctl->ticket_tu = 0;
    }
}

// value of v[j] once it is published; false if the wait gave up
__device__ __forceinline__ bool await_value(const double *v, int j, const SolveArgs &a, int site,
                                            int row, double &out)
{
    unsigned long long b = ld_relaxed_u64(v + j);
    long long it = 0;
    while (b == kSentinel) {
        // the shared status word is read only every 64 polls: thousands of
        // waiting lanes polling one address would queue on its L2 slice
        if (++it > a.spin_limit || ((it & 63) == 0 && ld_volatile(&a.ctl->status))) {
            set_status(a.ctl, GBLU_ERR_DEVICE_TIMEOUT);
            a.ctl->where = site;
            a.ctl->where_k = row;
            return false;
        }
        __nanosleep(32);
        b = ld_relaxed_u64(v + j);
    }
    out = __longlong_as_double((long long)b);
    return true;
}

// ---------------------------------------------------------------------------
// Sparse part of the two solves (Algorithm 2), by row blocks: a block is at
// most 32 consecutive rows f..l-1 whose diagonal block is dense (the rows of
// one supernode of L forward, of U backward).  One warp per row sums the
// row's entries outside its block (lanes over entries, waiting for each
// needed value to be published) and publishes that sum; the row that comes
// last in its block (the last row forward, the first backward) then gathers
// the block's sums and solves the dense diagonal block with shuffles, lane q
// holding row f+q, and publishes the block's values.  The chain of dependent
// steps is a chain of blocks, not of rows.  Values are published by
// overwriting a sentinel.  The arithmetic does not depend on when inputs
// arrive, so level launches (sums, then block finishes) and the sync-free
// launch give identical bits.
constexpr int kBR = kSolveBlockRows;

// forward: sum over the entries of row i outside its block (all but its last q)
// v[j] for four columns at once: one relaxed load each in flight, then a
// bounded wait on those still holding the sentinel
__device__ __forceinline__ bool fetch4(const double *v, const int (&j)[4], bool wait, const SolveArgs &a, int site,
                                       int row, double (&out)[4])
{
    if (!wait) {
#pragma unroll
        for (int u = 0; u < 4; u++) out[u] = __ldcg(v + j[u]);
        return true;
    }
    unsigned long long b[4];
#pragma unroll
    for (int u = 0; u < 4; u++) b[u] = ld_relaxed_u64(v + j[u]);
    bool ok = true;
#pragma unroll
    for (int u = 0; u < 4; u++) {
        if (b[u] != kSentinel) out[u] = __longlong_as_double((long long)b[u]);
        else if (ok) ok = await_value(v, j[u], a, site, row, out[u]);
    }
    return ok;
}

__device__ __forceinline__ bool lrow_ext(const SolveArgs &a, int i, int q, int lane, bool wait, double &s)
{
    const int64_t rb = __ldg(a.Lrp + i), re = __ldg(a.Lrp + i + 1) - q;
    double acc = 0.0;
    bool ok = true;
    int64_t e = rb + lane;
    // four entries per lane in flight, applied in the same order as one by one
    for (; e + 96 < re && ok; e += 128) {
        int j[4];
        double lv[4], yv[4];
#pragma unroll
        for (int u = 0; u < 4; u++) j[u] = __ldg(a.Lcol + e + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; u++) lv[u] = __ldg(a.LUx + __ldg(a.Lslot + e + 32 * u));
        ok = fetch4(a.y, j, wait, a, 3, i, yv);
#pragma unroll
        for (int u = 0; u < 4; u++) acc = fma(lv[u], yv[u], acc);
    }
    for (; e < re; e += 32) {
        const int j = __ldg(a.Lcol + e);
        double yj = 0.0;
        if (!wait) yj = __ldcg(a.y + j);
        else if (ok) ok = await_value(a.y, j, a, 3, i, yj);
        acc = fma(__ldg(a.LUx + __ldg(a.Lslot + e)), yj, acc);
    }
    s = warp_sum(acc);
    return __all_sync(kFull, ok);
}

// forward block finish: lane p < w holds e = the outside sum of row f+p
// the block's unit lower triangle: lane p < w holds row f+p's entries
// L(f+p, f .. f+p-1), its last p entries (loaded before the block's values
// are awaited, off the dependency chain)
__device__ __forceinline__ void lblock_load(const SolveArgs &a, int f, int w, int lane, double (&tv)[kBR - 1])
{
    const int64_t rend = lane < w ? __ldg(a.Lrp + f + lane + 1) - lane : 0;
#pragma unroll
    for (int d = 0; d < kBR - 1; d++)
        tv[d] = (d < lane && lane < w) ? __ldg(a.LUx + __ldg(a.Lslot + rend + d)) : 0.0;
}

// forward block finish: lane p < w holds e = the outside sum of row f+p
__device__ __forceinline__ void lblock_solve(const SolveArgs &a, int f, int w, int lane, double e,
                                             const double (&tv)[kBR - 1])
{
    double v = lane < w ? __ldg(a.b + __ldg(a.piv + f + lane)) - e : 0.0;
#pragma unroll
    for (int d = 0; d < kBR - 1; d++) {
        if (d < w - 1) {
            const double yd = __shfl_sync(kFull, v, d);
            if (lane > d && lane < w) v = fma(-tv[d], yd, v);
        }
    }
    if (lane < w) st_relaxed_f64(a.y + f + lane, v);
}

__device__ __forceinline__ void lblock_finish(const SolveArgs &a, int f, int w, int lane, double e)
{
    double tv[kBR - 1];
    lblock_load(a, f, w, lane, tv);
    lblock_solve(a, f, w, lane, e, tv);
}

// backward: sum over the entries of row i outside its block (all but its
// first w-1-q), from the last column down
__device__ __forceinline__ bool urow_ext(const SolveArgs &a, int i, int q, int w, int lane, bool wait,
                                         double &s)
{
    // entries in the trailing block's columns were summed into far[i] already
    const int64_t rb = __ldg(a.Urp + i) + (w - 1 - q), re = a.ufar ? __ldg(a.ufar + i) : __ldg(a.Urp + i + 1);
    double acc = 0.0;
    bool ok = true;
    int64_t e = re - 1 - lane;
    // four entries per lane in flight, applied in the same order as one by one
    for (; e - 96 >= rb && ok; e -= 128) {
        int j[4];
        double uv[4], zv[4];
#pragma unroll
        for (int u = 0; u < 4; u++) j[u] = __ldg(a.Ucol + e - 32 * u);
#pragma unroll
        for (int u = 0; u < 4; u++) uv[u] = __ldg(a.LUx + __ldg(a.Uslot + e - 32 * u));
        ok = fetch4(a.z, j, wait, a, 4, i, zv);
#pragma unroll
        for (int u = 0; u < 4; u++) acc = fma(uv[u], zv[u], acc);
    }
    for (; e >= rb; e -= 32) {
        const int j = __ldg(a.Ucol + e);
        double zj = 0.0;
        if (!wait) zj = __ldcg(a.z + j);
        else if (ok) ok = await_value(a.z, j, a, 4, i, zj);
        acc = fma(__ldg(a.LUx + __ldg(a.Uslot + e)), zj, acc);
    }
    s = warp_sum(acc);
    if (a.ufar) s += __ldcg(a.far + i);
    return __all_sync(kFull, ok);
}

// the block's upper triangle: lane p < w holds row f+p's entries
// U(f+p, f+p+1 .. f+w-1) (its first w-1-p entries) and the reciprocal of
// its diagonal, computed by every lane at once (a division per step of the
// substitution would sit on the dependency chain)
__device__ __forceinline__ void ublock_load(const SolveArgs &a, int f, int w, int lane, double (&tu)[kBR], double &rd)
{
    const int64_t rbeg = lane < w ? __ldg(a.Urp + f + lane) - lane - 1 : 0;
#pragma unroll
    for (int d = 0; d < kBR; d++)
        tu[d] = (lane < d && d < w) ? __ldg(a.LUx + __ldg(a.Uslot + rbeg + d)) : 0.0;
    rd = lane < w ? 1.0 / __ldg(a.LUx + __ldg(a.Udiag + f + lane)) : 1.0;
}

// backward block finish: lane p < w holds e = the outside sum of row f+p
__device__ __forceinline__ void ublock_solve(const SolveArgs &a, int f, int w, int lane, double e,
                                             const double (&tu)[kBR], double rd)
{
    double v = lane < w ? __ldcg(a.y + f + lane) - e : 0.0, zl = 0.0;
#pragma unroll
    for (int d = kBR - 1; d >= 0; d--) {
        if (d < w) {
            const double zd = __shfl_sync(kFull, v, d) * __shfl_sync(kFull, rd, d);
            if (lane == d) zl = zd;
            if (lane < d) v = fma(-tu[d], zd, v);
        }
    }
    if (lane < w) {
        st_relaxed_f64(a.z + f + lane, zl);
        a.x[__ldg(a.Q + f + lane)] = zl;
    }
}

__device__ __forceinline__ void ublock_finish(const SolveArgs &a, int f, int w, int lane, double e)
{
    double tu[kBR], rd;
    ublock_load(a, f, w, lane, tu, rd);
    ublock_solve(a, f, w, lane, e, tu, rd);
}

// Batches (gblu_solve_batch): the same kernels over nsets right-hand sides
// and factor value sets; set s reads its values at LUx + s*lu_stride and
// its vectors at b + s*b_stride, x + s*x_stride, y/z/ext + s*v_stride.
__device__ __forceinline__ SolveArgs set_view(const SolveArgs &a, int s)
{
    SolveArgs v = a;
    v.LUx = a.LUx + (int64_t)s * a.lu_stride;
    v.b = a.b + (int64_t)s * a.b_stride;
    v.x = a.x + (int64_t)s * a.x_stride;
    v.y = a.y + (int64_t)s * a.v_stride;
    v.z = a.z + (int64_t)s * a.v_stride;
    v.ext = a.ext + (int64_t)s * a.v_stride;
    if (a.far) v.far = a.far + (int64_t)s * a.v_stride;
    return v;
}

// level mode, first launch of a level: every row of the level stores its
// outside sum (its inputs are final: earlier launches)
__device__ __forceinline__ void lsolve_level_row(const SolveArgs &a, int t, int lane)
{
    const int i = __ldg(a.rows + t), b = __ldg(a.rb + i);
    double s;
    lrow_ext(a, i, i - __ldg(a.bs + b), lane, false, s);
    if (lane == 0) a.ext[i] = s;
}

__device__ __forceinline__ void usolve_level_row(const SolveArgs &a, int t, int lane)
{
    const int i = __ldg(a.rows + t), b = __ldg(a.rb + i);
    const int f = __ldg(a.bs + b), w = __ldg(a.bs + b + 1) - f;
    double s;
    urow_ext(a, i, i - f, w, lane, false, s);
    if (lane == 0) a.ext[i] = s;
}

// level mode, second launch of a level: one warp per block (a.rows = block ids)
__device__ __forceinline__ void lsolve_finish_block(const SolveArgs &a, int t, int lane)
{
    const int b = __ldg(a.rows + t), f = __ldg(a.bs + b), w = __ldg(a.bs + b + 1) - f;
    lblock_finish(a, f, w, lane, lane < w ? __ldcg(a.ext + f + lane) : 0.0);
}

__device__ __forceinline__ void usolve_finish_block(const SolveArgs &a, int t, int lane)
{
    const int b = __ldg(a.rows + t), f = __ldg(a.bs + b), w = __ldg(a.bs + b + 1) - f;
    ublock_finish(a, f, w, lane, lane < w ? __ldcg(a.ext + f + lane) : 0.0);
}

// kernels of the level launches; a batch puts the set in blockIdx.y
#define GBLU_WARP_KERNEL(name, body)                                                             \
    template <bool kBatch>                                                                      \
    __global__ void __launch_bounds__(kSolveWarpsPerBlock * 32) name(SolveArgs a)               \
    {                                                                                           \
        const int t = blockIdx.x * kSolveWarpsPerBlock + (threadIdx.x >> 5), lane = threadIdx.x & 31; \
        if (t >= a.nrows) return;                                                               \
        if (kBatch) body(set_view(a, blockIdx.y), t, lane);                                     \
        else body(a, t, lane);                                                                  \
    }
GBLU_WARP_KERNEL(lsolve_level_kernel, lsolve_level_row)
GBLU_WARP_KERNEL(usolve_level_kernel, usolve_level_row)
GBLU_WARP_KERNEL(lsolve_finish_kernel, lsolve_finish_block)
GBLU_WARP_KERNEL(usolve_finish_kernel, usolve_finish_block)
#undef GBLU_WARP_KERNEL

// sync-free: a.rows[0..nrows) = rows in a topological order (blocks by
// level, the finishing row of each block last), handed out by ticket; in a
// batch ticket t is row ticket t / nsets of set t % nsets.  true = stop.
__device__ __forceinline__ bool lsolve_sf_row(const SolveArgs &a, int t, int lane)
{
    const int i = __ldg(a.rows + t), b = __ldg(a.rb + i);
    const int f = __ldg(a.bs + b), w = __ldg(a.bs + b + 1) - f, q = i - f;
    double s;
    if (q < w - 1) {
        if (!lrow_ext(a, i, q, lane, true, s)) return true;
        if (lane == 0) st_relaxed_f64(a.ext + i, s);
        return false;
    }
    // the last row finishes the block; its triangle is loaded first
    double tv[kBR - 1];
    lblock_load(a, f, w, lane, tv);
    if (!lrow_ext(a, i, q, lane, true, s)) return true;
    double e = s;
    bool ok = true;
    if (lane < w - 1) ok = await_value(a.ext, f + lane, a, 5, f + lane, e);
    if (!__all_sync(kFull, ok)) return true;
    lblock_solve(a, f, w, lane, e, tv);
    return false;
}

__device__ __forceinline__ bool usolve_sf_row(const SolveArgs &a, int t, int lane)
{
    const int i = __ldg(a.rows + t), b = __ldg(a.rb + i);
    const int f = __ldg(a.bs + b), w = __ldg(a.bs + b + 1) - f, q = i - f;
    double s;
    if (q > 0) {
        if (!urow_ext(a, i, q, w, lane, true, s)) return true;
        if (lane == 0) st_relaxed_f64(a.ext + i, s);
        return false;
    }
    // the first row finishes the block; its triangle is loaded first
    double tu[kBR], rd;
    ublock_load(a, f, w, lane, tu, rd);
    if (!urow_ext(a, i, q, w, lane, true, s)) return true;
    double e = s;
    bool ok = true;
    if (lane >= 1 && lane < w) ok = await_value(a.ext, f + lane, a, 6, f + lane, e);
    if (!__all_sync(kFull, ok)) return true;
    ublock_solve(a, f, w, lane, e, tu, rd);
    return false;
}

#define GBLU_SYNCFREE_KERNEL(name, body, tick)                                                   \
    template <bool kBatch>                                                                      \
    __global__ void __launch_bounds__(kSolveWarpsPerBlock * 32) name(SolveArgs a)               \
    {                                                                                           \
        const int lane = threadIdx.x & 31;                                                      \
        const int total = kBatch ? a.nrows * a.nsets : a.nrows;                                 \
        for (;;) {                                                                              \
            int t = 0;                                                                          \
            if (lane == 0) t = atomicAdd(&a.ctl->tick, 1);                                      \
            t = __shfl_sync(kFull, t, 0);                                                       \
            if (t >= total) break;                                                              \
            const bool stop = kBatch ? body(set_view(a, t % a.nsets), t / a.nsets, lane)        \
                                     : body(a, t, lane);                                        \
            if (stop) break;                                                                    \
        }                                                                                       \
    }
GBLU_SYNCFREE_KERNEL(lsolve_syncfree_kernel, lsolve_sf_row, ticket_l)
GBLU_SYNCFREE_KERNEL(usolve_syncfree_kernel, usolve_sf_row, ticket_u)
#undef GBLU_SYNCFREE_KERNEL

// Several handles of different patterns in one launch per triangle: sets[s]
// is handle s's whole sparse triangle (rows in its ticket order); ticket t
// is row ticket order[t].task of set order[t].set.  Every set's rows keep
// their order, so a row only waits on rows with smaller tickets.
template <bool kLower>
__global__ void __launch_bounds__(kSolveWarpsPerBlock * 32)
solve_multi_kernel(const SolveArgs *sets, const SetTask *order, int total, int32_t *ticket)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(ticket, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= total) break;
        const SetTask o = order[t];
        const SolveArgs a = sets[o.set];
        const bool stop = kLower ? lsolve_sf_row(a, o.task, lane) : usolve_sf_row(a, o.task, lane);
        if (stop) break;
    }
}

// the sentinel fill of begin_solve_kernel for every set (blockIdx.y = set)
__global__ void begin_multi_solve_kernel(const SolveArgs *lo, const SolveArgs *up, int32_t *tickets)
{
    const double sent = __longlong_as_double((long long)kSentinel);
    const SolveArgs &a = lo[blockIdx.y];
    double *eu = up[blockIdx.y].ext;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        a.y[i] = sent;
        a.z[i] = sent;
        a.ext[i] = sent;
        eu[i] = sent;
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        tickets[0] = 0;
        tickets[1] = 0;
    }
}

// ---------------------------------------------------------------------------
// Trailing block of the structure-adaptive solve (Section V-B, Algorithm 6).
// The paper cuts the trailing rows [p0, n) into trapezoid slices, each a
// rectangular product with the final part of the vector followed by a small
// triangle.  Here a slice is kTrailRows = 32 rows, one warp (lane q holds
// row p0 + 32 I + q of slice I), and the slices run sync-free: slice I takes
// the 32-column blocks J of its rectangle as their values are published,
// one 32 x 32 tile at a time (staged in shared memory from the factor's
// column storage before the wait, then 32 multiply-adds per lane into four
// accumulators), and finishes with its diagonal triangle by shuffles.  The
// chain of dependent steps is the chain of slices, not of rows.  Values are
// published by overwriting the solve's NaN sentinel, as in the row blocks.
// Forward, the rows' entries before p0 (final before the block starts) are
// summed first by a fully parallel launch; backward, the block comes first
// and the sums of rows < p0 over its columns follow in a parallel launch.
constexpr int kTB = kTrailRows;
constexpr int kTileLd = kTB + 1;      // padded leading dimension of a tile
constexpr int kTrailWarps = 4;        // warps per slice (one CTA)

// out = sum over CSR entries [e0, e1) of LUx[slot[e]] * v[col[e]], one warp,
// four entries per lane in flight
__device__ __forceinline__ double row_dot(const double *LUx, const int32_t *col, const int32_t *slot,
                                          const double *v, int64_t e0, int64_t e1, int lane)
{
    double s0 = 0.0, s1 = 0.0;
    int64_t e = e0 + lane;
    for (; e + 96 < e1; e += 128) {
        const int c0 = __ldg(col + e), c1 = __ldg(col + e + 32), c2 = __ldg(col + e + 64), c3 = __ldg(col + e + 96);
        const int q0 = __ldg(slot + e), q1 = __ldg(slot + e + 32), q2 = __ldg(slot + e + 64), q3 = __ldg(slot + e + 96);
        const double v0 = __ldcg(v + c0), v1 = __ldcg(v + c1), v2 = __ldcg(v + c2), v3 = __ldcg(v + c3);
        s0 = fma(__ldg(LUx + q0), v0, s0);
        s1 = fma(__ldg(LUx + q1), v1, s1);
        s0 = fma(__ldg(LUx + q2), v2, s0);
        s1 = fma(__ldg(LUx + q3), v3, s1);
    }
    for (; e < e1; e += 32) s0 = fma(__ldg(LUx + __ldg(slot + e)), __ldcg(v + __ldg(col + e)), s0);
    return warp_sum(s0 + s1);
}

// forward, rows i >= p0: ext[i] = L(i, columns < p0) y
template <bool kBatch>
__global__ void __launch_bounds__(kSolveWarpsPerBlock * 32) ltrail_rect_kernel(SolveArgs a0, TrailArgs t)
{
    const int i = t.p0 + blockIdx.x * kSolveWarpsPerBlock + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= t.n) return;
    const SolveArgs a = kBatch ? set_view(a0, blockIdx.y) : a0;
    const double s = row_dot(a.LUx, a.Lcol, a.Lslot, a.y, __ldg(a.Lrp + i), __ldg(t.rows + (i - t.p0)), lane);
    if (lane == 0) a.ext[i] = s;
}

// backward, rows i < p0: far[i] = U(i, columns >= p0) z
template <bool kBatch>
__global__ void __launch_bounds__(kSolveWarpsPerBlock * 32) utrail_far_kernel(SolveArgs a0, TrailArgs t)
{
    const int i = blockIdx.x * kSolveWarpsPerBlock + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= t.p0) return;
    const SolveArgs a = kBatch ? set_view(a0, blockIdx.y) : a0;
    const double s = row_dot(a.LUx, a.Ucol, a.Uslot, a.z, __ldg(t.rows + i), __ldg(a.Urp + i + 1), lane);
    if (lane == 0) a.far[i] = s;
}

// Stage the tile of slice I (rows i0 = p0 + 32 I ...) and column block J:
// tile[c * kTileLd + r] = F(i0 + r, j0 + c), zero where the factor has no
// entry.  Column j's entries with rows in slice I are [seg[j][I],
// seg[j][I+1]) from base(j); lane c first reads column j0 + c's bounds.
// false (tile untouched): the slice's rows have no entry in these columns.
__device__ __forceinline__ bool trail_stage(double *tile, const double *LUx, const TrailArgs &t, bool lower,
                                            int I, int J, int lane)
{
    const int i0 = t.p0 + kTB * I, j0 = t.p0 + kTB * J;
    const int wj = min(kTB, t.n - j0);
    int s = 0, e = 0;
    int64_t base = 0;
    if (lane < wj) {
        const int j = j0 + lane;
        const int32_t *sg = t.seg + (int64_t)(j - t.p0) * (t.nb + 1);
        s = __ldg(sg + I);
        e = __ldg(sg + I + 1);
        base = __ldg(t.LUp + j) + (lower ? __ldg(t.nU + j) : 0);
    }
    if (!__any_sync(kFull, e > s)) return false;
    for (int idx = lane; idx < kTB * kTileLd; idx += 32) tile[idx] = 0.0;
    __syncwarp();
    // sixteen columns' loads in flight at a time (lane q: entry q of each
    // column's segment), then their scatter into the tile
#pragma unroll
    for (int h = 0; h < kTB; h += 16) {
        double v[16];
        int r[16];
#pragma unroll
        for (int u = 0; u < 16; u++) {
            const int c = h + u;
            const int sc = __shfl_sync(kFull, s, c), ec = __shfl_sync(kFull, e, c);
            const int64_t bc = __shfl_sync(kFull, base, c);
            const bool has = c < wj && sc + lane < ec;
            r[u] = has ? __ldg(t.LUi + bc + sc + lane) - i0 : -1;
            v[u] = has ? __ldg(LUx + bc + sc + lane) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 16; u++)
            if (r[u] >= 0) tile[(h + u) * kTileLd + r[u]] = v[u];
    }
    __syncwarp();
    return true;
}

// One slice per CTA of kTrailWarps warps: warp w takes the column blocks
// J = w, w + 4, ... of the slice's rectangle (forward: J < I ascending;
// backward: J > I descending), staging the next block's tile before it
// waits for the current one's values; its four partial sums per row go to
// shared memory, and warp 0 adds them in a fixed order (so the result does
// not depend on timing) and finishes the slice's triangle.  true = a wait
// gave up.
template <bool kLower>
__device__ bool trail_slice(const SolveArgs &a, const TrailArgs &t, int I, double *wt, double *dtile, double *part,
                            int *s_bad, int warp, int lane)
{
    const int i0 = t.p0 + kTB * I, w = min(kTB, t.n - i0), i = i0 + lane;
    if (warp == 0 && !trail_stage(dtile, a.LUx, t, kLower, I, I, lane))   // off the critical path
        for (int idx = lane; idx < kTB * kTileLd; idx += 32) dtile[idx] = 0.0;
    // this warp's blocks: J(m) = first + step * m while in range
    const int first = kLower ? warp : t.nb - 1 - warp, step = kLower ? kTrailWarps : -kTrailWarps;
    auto in_range = [&](int J) { return kLower ? J < I : J > I; };
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
    bool ok = true;
    int J = first;
    bool have = in_range(J) && trail_stage(wt, a.LUx, t, kLower, I, J, lane);
    for (int m = 0; in_range(J) && ok; m++) {
        const int Jn = J + step;
        double *cur = wt + (m & 1) * (kTB * kTileLd), *nxt = wt + ((m + 1) & 1) * (kTB * kTileLd);
        const bool have_n = in_range(Jn) && trail_stage(nxt, a.LUx, t, kLower, I, Jn, lane);
        if (have) {
            const int j0 = t.p0 + kTB * J, wj = min(kTB, t.n - j0);
            double vq = 0.0;
            bool got = true;
            if (lane < wj) got = await_value(kLower ? a.y : a.z, j0 + lane, a, kLower ? 7 : 8, i0, vq);
            ok = __all_sync(kFull, got);
            if (ok) {
#pragma unroll
                for (int c = 0; c < kTB; c += 4) {   // columns past wj hold zero tiles and vq = 0
                    acc0 = fma(cur[(c + 0) * kTileLd + lane], __shfl_sync(kFull, vq, c + 0), acc0);
                    acc1 = fma(cur[(c + 1) * kTileLd + lane], __shfl_sync(kFull, vq, c + 1), acc1);
                    acc2 = fma(cur[(c + 2) * kTileLd + lane], __shfl_sync(kFull, vq, c + 2), acc2);
                    acc3 = fma(cur[(c + 3) * kTileLd + lane], __shfl_sync(kFull, vq, c + 3), acc3);
                }
            }
            __syncwarp();
        }
        have = have_n;
        J = Jn;
    }
    part[warp * 32 + lane] = (acc0 + acc1) + (acc2 + acc3);
    if (!ok && lane == 0) *s_bad = 1;
    __syncthreads();
    if (*s_bad) return true;
    if (warp == 0) {
        double sum = 0.0;
#pragma unroll
        for (int q = 0; q < kTrailWarps; q++) sum += part[q * 32 + lane];
        if (kLower) {
            double v = 0.0;
            if (lane < w) v = __ldg(a.b + __ldg(a.piv + i)) - __ldcg(a.ext + i) - sum;
            for (int c = 0; c < w - 1; c++) {
                const double yc = __shfl_sync(kFull, v, c);
                if (lane > c && lane < w) v = fma(-dtile[c * kTileLd + lane], yc, v);
            }
            if (lane < w) st_relaxed_f64(a.y + i, v);
        } else {
            double v = 0.0, zl = 0.0;
            if (lane < w) v = __ldcg(a.y + i) - sum;
            // reciprocals of the diagonal by every lane at once, off the chain
            const double rd = lane < w ? 1.0 / dtile[lane * kTileLd + lane] : 1.0;
            for (int c = w - 1; c >= 0; c--) {
                const double zc = __shfl_sync(kFull, v, c) * __shfl_sync(kFull, rd, c);
                if (lane == c) zl = zc;
                if (lane < c) v = fma(-dtile[c * kTileLd + lane], zc, v);
            }
            if (lane < w) {
                st_relaxed_f64(a.z + i, zl);
                a.x[__ldg(a.Q + i)] = zl;
            }
        }
    }
    __syncthreads();   // tiles and partial sums are reused by the next slice
    return false;
}

// slices handed out by ticket (one per CTA) in their dependency order
// (forward ascending, backward descending); in a batch ticket t is slice
// t / nsets of set t % nsets, so a CTA only waits on smaller tickets
template <bool kLower, bool kBatch>
__global__ void __launch_bounds__(kTrailWarps * 32) trail_slice_kernel(SolveArgs a0, TrailArgs t)
{
    extern __shared__ __align__(16) double tsmem[];
    __shared__ double part[kTrailWarps * 32];
    __shared__ int s_k, s_bad;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *dtile = tsmem, *wt = tsmem + kTB * kTileLd + warp * (2 * kTB * kTileLd);
    const int nsets = kBatch ? a0.nsets : 1;
    const int total = t.nb * nsets;
    if (threadIdx.x == 0) s_bad = 0;
    for (;;) {
        if (threadIdx.x == 0) s_k = atomicAdd(kLower ? &a0.ctl->ticket_tl : &a0.ctl->ticket_tu, 1);
        __syncthreads();
        const int k = s_k;
        __syncthreads();
        if (k >= total) break;
        const int s = k % nsets, q = k / nsets;
        const SolveArgs a = kBatch ? set_view(a0, s) : a0;
        if (trail_slice<kLower>(a, t, kLower ? q : t.nb - 1 - q, wt, dtile, part, &s_bad, warp, lane)) break;
    }
}

// ---------------------------------------------------------------------------
// rvec (optional): receives r = b - A x
__global__ void residual_kernel(int32_t n, const int64_t *Arp, const int32_t *Acol,
                                const int32_t *Aslot, const double *Ax, const double *b,
                                const double *x, double *partial, double *rvec)
{
    __shared__ double sr[8], sa[8], sx[8];
    double rmax = 0.0, amax = 0.0, xmax = 0.0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = blockIdx.x * 8 + warp; i < n; i += gridDim.x * 8) {
        double s = 0.0, as = 0.0;
        for (int64_t e = Arp[i] + lane; e < Arp[i + 1]; e += 32) {
            const double v = Ax[Aslot[e]];
            s = fma(v, x[Acol[e]], s);
            as += fabs(v);
        }
        s = warp_sum(s);
        as = warp_sum(as);
        if (rvec && lane == 0) rvec[i] = b[i] - s;
        rmax = max_nan(rmax, fabs(b[i] - s));
        amax = max_nan(amax, as);
        xmax = max_nan(xmax, fabs(x[i]));
    }
    if (lane == 0) { sr[warp] = rmax; sa[warp] = amax; sx[warp] = xmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; w++) { rmax = max_nan(rmax, sr[w]); amax = max_nan(amax, sa[w]); xmax = max_nan(xmax, sx[w]); }
        partial[3 * blockIdx.x + 0] = rmax;
        partial[3 * blockIdx.x + 1] = amax;
        partial[3 * blockIdx.x + 2] = xmax;
    }
}

__global__ void residual_final_kernel(const double *partial, int nblocks, double *out)
{
    double r = 0.0, a = 0.0, x = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += 32) {
        r = max_nan(r, partial[3 * i]);
        a = max_nan(a, partial[3 * i + 1]);
        x = max_nan(x, partial[3 * i + 2]);
    }
    r = warp_max(r);
    a = warp_max(a);
    x = warp_max(x);
    if (threadIdx.x == 0) {
        out[0] = (a > 0.0 && x > 0.0) ? r / (a * x) : r;
        out[1] = r;
        out[2] = a;
        out[3] = x;
    }
}

// mixed precision: single-precision factor values widened for the FP64
// solves of iterative refinement, and the correction step x += d
// out[k] = in[src[k]] * scale[k] (src == nullptr: in[k]); the per-step
// application of a static row permutation and scaling to values and vectors
__global__ void gather_scale_kernel(int64_t m, const int32_t *src, const double *scale, const double *in,
                                    double *out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const double v = __ldg(in + (src ? __ldg(src + k) : k));
        out[k] = scale ? v * __ldg(scale + k) : v;
    }
}

// Pivot verification of a single-precision re-factorization, in double.
// Column k's single-precision pivot d carries a rounding error of the order
// of u32 * S_k, where S_k = |d| + sum_j |L(k,j)| |U(j,k)| is the magnitude
// summed into it (u32 = 2^-24); the max m = |d| max|L(:,k)| is close to its
// double value.  The column passes only if the threshold test still holds
// with d moved towards zero by kF32Margin * S_k and m enlarged by the same
// relative amount: then the double-precision check of the same step passes
// too, up to that estimate.  Any other column counts as failed, so that the
// double-precision re-factorization (its check, and its restart) decides.
// One warp per column; row k of L comes from the row-wise copy, U(j,k) from
// a bisection in the column's sorted U rows.
constexpr double kF32Margin = 1.0 / 4096.0;

__global__ void f32_verify_kernel(int32_t n, const int64_t *LUp, const int32_t *LUi, const int32_t *nU,
                                  const float *LUx, const int64_t *Lrp, const int32_t *Lcol,
                                  const int32_t *Lslot, double eps, DevCtl *ctl)
{
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n; k += warps) {
        const int64_t beg = __ldg(LUp + k), end = __ldg(LUp + k + 1);
        const int nu = __ldg(nU + k);
        const double d = (double)__ldg(LUx + beg + nu - 1);
        double lmax = 0.0, sum = 0.0;
        for (int64_t e = beg + nu + lane; e < end; e += 32) lmax = max_nan(lmax, fabs((double)__ldg(LUx + e)));
        for (int64_t e = __ldg(Lrp + k) + lane; e < __ldg(Lrp + k + 1); e += 32) {
            const int j = __ldg(Lcol + e);
            int lo = 0, hi = nu - 2;   // the U rows above the diagonal, ascending
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(LUi + beg + mid) < j) lo = mid + 1;
                else hi = mid;
            }
            if (hi >= 0 && lo == hi && __ldg(LUi + beg + lo) == j)
                sum += fabs((double)__ldg(LUx + __ldg(Lslot + e))) * fabs((double)__ldg(LUx + beg + lo));
        }
        lmax = warp_max(lmax);
        sum = warp_sum(sum);
        if (lane == 0) {
            const double S = fabs(d) + sum;
            const double m = fabs(d) * lmax;
            const bool ok = d != 0.0 && isfinite(d) && isfinite(S) && !(m != m) &&
                            fabs(d) - kF32Margin * S >= eps * m * (1.0 + kF32Margin);
            if (!ok) {
                atomicExch(&ctl->interrupted, 1);
                atomicMin(&ctl->first_bad, k);
            }
        }
    }
}

__global__ void widen_kernel(const float *src, double *dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

__global__ void axpy_kernel(double *x, const double *d, int32_t n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] += d[i];
}

}  // namespace

// After a restart that kept every pivot, the factor structure is the old
// one (the pattern is fixed by the pattern of A and the pivot order), so the
// recomputed columns only move their values from the pool into their
// canonical slots.  One warp per restarted step k: the pool holds U entries
// as step ids and L entries as original rows; each goes to the slot of its
// step in the sorted canonical column.  Any mismatch sets *bad (the caller
// then rebuilds the structure instead).
__global__ void pool_scatter_kernel(const int32_t *seq, int32_t nseq, const int64_t *cbeg, const int32_t *cnu,
                                    const int32_t *cnl, const int32_t *prow, const int64_t *LUp,
                                    const int32_t *LUi, const int32_t *pinv, int32_t n, double *vals, int32_t *bad)
{
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int t = w; t < nseq; t += nw) {
        const int k = __ldg(seq + t);
        const int64_t b = cbeg[k];
        const int nu = cnu[k], nl = cnl[k];
        const int64_t lo = __ldg(LUp + k);
        const int len = (int)(__ldg(LUp + k + 1) - lo);
        if (nu + nl != len) {
            if (lane == 0) atomicExch(bad, 1);
            continue;
        }
        for (int e = lane; e < len; e += 32) {
            const int r = prow[b + e];
            const int s = e < nu ? r : ((unsigned)r < (unsigned)n ? __ldg(pinv + r) : -1);
            int a = 0, z = len;   // first slot with LUi >= s
            while (a < z) {
                const int m = (a + z) >> 1;
                if (__ldg(LUi + lo + m) < s) a = m + 1;
                else z = m;
            }
            if (s < 0 || a >= len || __ldg(LUi + lo + a) != s) atomicExch(bad, 1);
            else vals[lo + a] = vals[b + e];
        }
    }
}

// ------------------------------------------------------------------ launchers
int launch_pool_scatter(const int32_t *seq, int32_t nseq, const int64_t *cbeg, const int32_t *cnu,
                        const int32_t *cnl, const int32_t *prow, const int64_t *LUp, const int32_t *LUi,
                        const int32_t *pinv, int32_t n, double *vals, int32_t *bad, void *stream)
{
    if (nseq <= 0) return 0;
    int grid = (nseq + 7) / 8;
    if (grid > 4096) grid = 4096;
    pool_scatter_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(seq, nseq, cbeg, cnu, cnl, prow, LUp, LUi, pinv, n,
                                                                 vals, bad);
    return (int)cudaGetLastError();
}

// Threshold pivoting at the first step whose check failed (Section II-A,
// the pivot choice of Algorithm 1).  The candidates of column k are its
// predicted pivot slot (step k) and its L rows (steps s > k), slot s standing
// for the row piv[s]; the column holds its values unnormalized (a failed
// check in no-stop mode).  The choice is the candidate of largest |x|, ties
// going to the row that comes first in the column order Q (smallest
// qinv[row]); a zero candidate is never chosen.  out[0] = the chosen slot's
// step (-1 when every candidate is zero), out[1] = 1 when a candidate is
// infinite or NaN.  One block.
__global__ void pivot_choice_kernel(const int64_t *LUp, const int32_t *LUi, const double *LUx, const int32_t *nU,
                                    const int32_t *piv, const int32_t *qinv, int32_t k, int32_t *out)
{
    __shared__ double s_a[32];
    __shared__ int s_q[32], s_s[32], s_bad[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t beg = LUp[k];
    const int len = (int)(LUp[k + 1] - beg);
    const int u = nU[k];
    double ba = 0.0;
    int bq = INT_MAX, bs = -1;
    bool bad = false;
    for (int i = u - 1 + (int)threadIdx.x; i < len; i += blockDim.x) {
        const double v = LUx[beg + i];
        if (!isfinite(v)) {
            bad = true;
            continue;
        }
        const double av = fabs(v);
        if (av == 0.0) continue;
        const int s = LUi[beg + i];
        const int q = qinv[piv[s]];
        if (av > ba || (av == ba && q < bq)) {
            ba = av;
            bq = q;
            bs = s;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double oa = __shfl_down_sync(0xffffffffu, ba, o);
        const int oq = __shfl_down_sync(0xffffffffu, bq, o);
        const int os = __shfl_down_sync(0xffffffffu, bs, o);
        if (oa > ba || (oa == ba && oq < bq)) {
            ba = oa;
            bq = oq;
            bs = os;
        }
    }
    const bool any_bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        s_a[warp] = ba;
        s_q[warp] = bq;
        s_s[warp] = bs;
        s_bad[warp] = any_bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int flag = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            flag |= s_bad[w];
            if (s_a[w] > ba || (s_a[w] == ba && s_q[w] < bq)) {
                ba = s_a[w];
                bq = s_q[w];
                bs = s_s[w];
            }
        }
        out[0] = bs;
        out[1] = flag;
    }
}

int launch_pivot_choice(const int64_t *LUp, const int32_t *LUi, const double *LUx, const int32_t *nU,
                        const int32_t *piv, const int32_t *qinv, int32_t k, int32_t *out, void *stream)
{
    pivot_choice_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(LUp, LUi, LUx, nU, piv, qinv, k, out);
    return (int)cudaGetLastError();
}

int launch_begin_tail(DevCtl *ctl, unsigned long long pool_base, void *stream)
{
    begin_tail_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(ctl, pool_base);
    return (int)cudaGetLastError();
}

// steps seq[0..nseq) start again; the row -> step map is cleared here and
// rebuilt from the kept steps by tail_pinv_kernel
__global__ void tail_repass_kernel(DevCtl *ctl, const int32_t *seq, int32_t nseq, int32_t n, int32_t *piv,
                                   int32_t *pinv, int32_t *done)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nseq; t += gridDim.x * blockDim.x) {
        const int k = seq[t];
        piv[k] = -1;
        done[k] = 0;
    }
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) pinv[r] = -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->tail_ticket = 0;
        ctl->tail_frontier = 0;
        ctl->tail_mispredict = INT_MAX;
        ctl->abort_tail = 0;
        ctl->status = 0;
        ctl->where = 0;
        ctl->where_k = -1;
    }
}

__global__ void tail_pinv_kernel(int32_t n, const int32_t *piv, int32_t *pinv)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int r = piv[k];
        if (r >= 0) pinv[r] = k;
    }
}

int launch_tail_repass(DevCtl *ctl, const int32_t *seq, int32_t nseq, int32_t n, int32_t *piv, int32_t *pinv,
                       int32_t *done, void *stream)
{
    const int m = nseq > n ? nseq : n;
    int g = (m + 255) / 256;
    g = g < 1 ? 1 : (g > 4096 ? 4096 : g);
    tail_repass_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(ctl, seq, nseq, n, piv, pinv, done);
    tail_pinv_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(n, piv, pinv);
    return (int)cudaGetLastError();
}

int launch_tail_init(int32_t n, const int32_t *restart_mask, const int32_t *piv_old,
                     int32_t *pinv, int32_t *piv, int32_t *done, int epoch, void *stream)
{
    const int grid = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    tail_init_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(n, restart_mask, piv_old, pinv, piv, done, epoch);
    return (int)cudaGetLastError();
}

int tail_setup()
{
    return (int)cudaFuncSetAttribute(tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kTailSmemBits / 8));
}

int launch_tail(const TailArgs &a, int grid, int epoch, void *stream)
{
    if (a.nseq <= 0) return 0;
    const size_t smem = a.bits_in_smem ? (size_t)((a.n + 31) >> 5) * sizeof(unsigned) : 0;
    tail_kernel<<<grid, kTailThreads, smem, (cudaStream_t)stream>>>(a, epoch);
    return (int)cudaGetLastError();
}

int launch_begin_solve(DevCtl *ctl, double *y, double *z, double *el, double *eu, int n, void *stream)
{
    int grid = (n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048;
    if (grid < 1) grid = 1;
    begin_solve_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(ctl, y, z, el, eu, n);
    return (int)cudaGetLastError();
}

// a.nsets > 1: a batch (set in blockIdx.y of the level launches, in the
// ticket of the sync-free launch)
int launch_lsolve(const SolveArgs &a, bool level_mode, int grid, void *stream)
{
    if (a.nrows <= 0) return 0;
    const bool batch = a.nsets > 1;
    const dim3 g((a.nrows + kSolveWarpsPerBlock - 1) / kSolveWarpsPerBlock, batch ? a.nsets : 1);
    cudaStream_t st = (cudaStream_t)stream;
    if (level_mode) {
        if (batch) lsolve_level_kernel<true><<<g, kSolveWarpsPerBlock * 32, 0, st>>>(a);
        else lsolve_level_kernel<false><<<g, kSolveWarpsPerBlock * 32, 0, st>>>(a);
    } else {
        if (batch) lsolve_syncfree_kernel<true><<<grid, kSolveWarpsPerBlock * 32, 0, st>>>(a);
        else lsolve_syncfree_kernel<false><<<grid, kSolveWarpsPerBlock * 32, 0, st>>>(a);
    }
    return (int)cudaGetLastError();
}

int launch_solve_finish(const SolveArgs &a, bool lower, void *stream)
{
    if (a.nrows <= 0) return 0;
    const bool batch = a.nsets > 1;
    const dim3 g((a.nrows + kSolveWarpsPerBlock - 1) / kSolveWarpsPerBlock, batch ? a.nsets : 1);
    cudaStream_t st = (cudaStream_t)stream;
    if (lower) {
        if (batch) lsolve_finish_kernel<true><<<g, kSolveWarpsPerBlock * 32, 0, st>>>(a);
        else lsolve_finish_kernel<false><<<g, kSolveWarpsPerBlock * 32, 0, st>>>(a);
    } else {
        if (batch) usolve_finish_kernel<true><<<g, kSolveWarpsPerBlock * 32, 0, st>>>(a);
        else usolve_finish_kernel<false><<<g, kSolveWarpsPerBlock * 32, 0, st>>>(a);
    }
    return (int)cudaGetLastError();
}

int launch_solve_multi(const SolveArgs *lo, const SolveArgs *up, int nsets, int max_n, const SetTask *order_l,
                       int total_l, const SetTask *order_u, int total_u, int grid, int32_t *tickets, void *stream)
{
    if (nsets <= 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    int gx = (max_n + 255) / 256;
    gx = gx < 1 ? 1 : (gx > 64 ? 64 : gx);
    begin_multi_solve_kernel<<<dim3(gx, nsets), 256, 0, st>>>(lo, up, tickets);
    solve_multi_kernel<true><<<grid, kSolveWarpsPerBlock * 32, 0, st>>>(lo, order_l, total_l, tickets);
    solve_multi_kernel<false><<<grid, kSolveWarpsPerBlock * 32, 0, st>>>(up, order_u, total_u, tickets + 1);
    return (int)cudaGetLastError();
}

int launch_usolve(const SolveArgs &a, bool level_mode, int grid, void *stream)
{
    if (a.nrows <= 0) return 0;
    const bool batch = a.nsets > 1;
    const dim3 g((a.nrows + kSolveWarpsPerBlock - 1) / kSolveWarpsPerBlock, batch ? a.nsets : 1);
    cudaStream_t st = (cudaStream_t)stream;
    if (level_mode) {
        if (batch) usolve_level_kernel<true><<<g, kSolveWarpsPerBlock * 32, 0, st>>>(a);
        else usolve_level_kernel<false><<<g, kSolveWarpsPerBlock * 32, 0, st>>>(a);
    } else {
        if (batch) usolve_syncfree_kernel<true><<<grid, kSolveWarpsPerBlock * 32, 0, st>>>(a);
        else usolve_syncfree_kernel<false><<<grid, kSolveWarpsPerBlock * 32, 0, st>>>(a);
    }
    return (int)cudaGetLastError();
}

int launch_trail(const SolveArgs &a, const TrailArgs &t, bool lower, int grid, void *stream)
{
    if (t.nb <= 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    const bool batch = a.nsets > 1;
    const int sets = batch ? a.nsets : 1;
    const size_t sm = (size_t)(2 * kTrailWarps + 1) * kTB * kTileLd * sizeof(double);
    const long long total = (long long)t.nb * sets;
    long long g = total;   // one slice per CTA
    if (g > grid) g = grid;
    if (g < 1) g = 1;
    if (lower) {
        const dim3 gr((t.n - t.p0 + kSolveWarpsPerBlock - 1) / kSolveWarpsPerBlock, sets);
        if (batch) {
            ltrail_rect_kernel<true><<<gr, kSolveWarpsPerBlock * 32, 0, st>>>(a, t);
            trail_slice_kernel<true, true><<<(unsigned)g, kTrailWarps * 32, sm, st>>>(a, t);
        } else {
            ltrail_rect_kernel<false><<<gr, kSolveWarpsPerBlock * 32, 0, st>>>(a, t);
            trail_slice_kernel<true, false><<<(unsigned)g, kTrailWarps * 32, sm, st>>>(a, t);
        }
    } else {
        const dim3 gr((t.p0 + kSolveWarpsPerBlock - 1) / kSolveWarpsPerBlock, sets);
        if (batch) {
            trail_slice_kernel<false, true><<<(unsigned)g, kTrailWarps * 32, sm, st>>>(a, t);
            if (t.p0 > 0) utrail_far_kernel<true><<<gr, kSolveWarpsPerBlock * 32, 0, st>>>(a, t);
        } else {
            trail_slice_kernel<false, false><<<(unsigned)g, kTrailWarps * 32, sm, st>>>(a, t);
            if (t.p0 > 0) utrail_far_kernel<false><<<gr, kSolveWarpsPerBlock * 32, 0, st>>>(a, t);
        }
    }
    return (int)cudaGetLastError();
}

int trail_setup(int *blocks_per_sm)
{
    const size_t sm = (size_t)(2 * kTrailWarps + 1) * kTB * kTileLd * sizeof(double);
    int a = 0, b = 0;
    cudaError_t e = cudaSuccess;
    for (auto f : {trail_slice_kernel<true, false>, trail_slice_kernel<false, false>, trail_slice_kernel<true, true>,
                   trail_slice_kernel<false, true>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, trail_slice_kernel<true, false>, kTrailWarps * 32, sm);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trail_slice_kernel<false, false>, kTrailWarps * 32, sm);
    *blocks_per_sm = a < b ? a : b;
    return (int)e;
}

int solve_syncfree_grid(int *grid)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int p[4] = {0, 0, 0, 0};
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p[0], lsolve_syncfree_kernel<false>,
                                                                  kSolveWarpsPerBlock * 32, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p[1], usolve_syncfree_kernel<false>,
                                                          kSolveWarpsPerBlock * 32, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p[2], lsolve_syncfree_kernel<true>,
                                                          kSolveWarpsPerBlock * 32, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p[3], usolve_syncfree_kernel<true>,
                                                          kSolveWarpsPerBlock * 32, 0);
    if (e != cudaSuccess) return (int)e;
    per = p[0];
    for (int i = 1; i < 4; i++) per = p[i] < per ? p[i] : per;
    *grid = sms * per;
    return 0;
}

int launch_f32_verify(int32_t n, const int64_t *LUp, const int32_t *LUi, const int32_t *nU, const float *LUx,
                      const int64_t *Lrp, const int32_t *Lcol, const int32_t *Lslot, double eps, DevCtl *ctl,
                      int grid, void *stream)
{
    f32_verify_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(n, LUp, LUi, nU, LUx, Lrp, Lcol, Lslot, eps, ctl);
    return (int)cudaGetLastError();
}

int launch_residual(int32_t n, const int64_t *Arp, const int32_t *Acol, const int32_t *Aslot,
                    const double *Ax, const double *b, const double *x, double *out,
                    double *partial, int nblocks, void *stream, double *rvec)
{
    residual_kernel<<<nblocks, 256, 0, (cudaStream_t)stream>>>(n, Arp, Acol, Aslot, Ax, b, x, partial, rvec);
    residual_final_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(partial, nblocks, out);
    return (int)cudaGetLastError();
}

int launch_gather_scale(int64_t m, const int32_t *src, const double *scale, const double *in, double *out,
                        void *stream)
{
    if (m <= 0) return 0;
    int64_t g = (m + 255) / 256;
    if (g > 8192) g = 8192;
    gather_scale_kernel<<<(unsigned)g, 256, 0, (cudaStream_t)stream>>>(m, src, scale, in, out);
    return (int)cudaGetLastError();
}

int launch_widen(const float *src, double *dst, int64_t n, void *stream)
{
    if (n <= 0) return 0;
    const int64_t g = (n + 255) / 256;
    widen_kernel<<<(unsigned)(g < 4096 ? g : 4096), 256, 0, (cudaStream_t)stream>>>(src, dst, n);
    return (int)cudaGetLastError();
}

int launch_axpy(double *x, const double *d, int32_t n, void *stream)
{
    if (n <= 0) return 0;
    const int g = (n + 255) / 256;
    axpy_kernel<<<g < 4096 ? g : 4096, 256, 0, (cudaStream_t)stream>>>(x, d, n);
    return (int)cudaGetLastError();
}

}  // namespace gblu
