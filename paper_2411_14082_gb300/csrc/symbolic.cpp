// Host-side symbolic work: input validation, elimination trees, the fill
// estimate of a first factorization and the fixed-pattern schedules.  No
// device code and no CUDA calls in this file.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <thread>

#include "gblu_internal.h"

namespace gblu {

int validate_pattern(int32_t n, const int32_t *Ap, const int32_t *Ai, std::string &err)
{
    if (n < 1) { err = "n must be >= 1"; return GBLU_ERR_INVALID_INPUT; }
    if (!Ap || !Ai) { err = "null pattern pointer"; return GBLU_ERR_INVALID_INPUT; }
    if (Ap[0] != 0) { err = "Ap[0] != 0"; return GBLU_ERR_INVALID_INPUT; }
    for (int32_t c = 0; c < n; c++)
        if (Ap[c + 1] < Ap[c]) { err = "Ap not non-decreasing at column " + std::to_string(c); return GBLU_ERR_INVALID_INPUT; }
    std::vector<int32_t> seen(n, -1);
    for (int32_t c = 0; c < n; c++) {
        for (int32_t p = Ap[c]; p < Ap[c + 1]; p++) {
            int32_t r = Ai[p];
            if (r < 0 || r >= n) { err = "row index out of range in column " + std::to_string(c); return GBLU_ERR_INVALID_INPUT; }
            if (seen[r] == c) { err = "duplicate entry (" + std::to_string(r) + "," + std::to_string(c) + ")"; return GBLU_ERR_INVALID_INPUT; }
            seen[r] = c;
        }
    }
    return GBLU_OK;
}

// Column elimination tree of B = A(:,Q): the elimination tree of B^T B,
// computed without forming B^T B (Section II-B: the ETree "is built from
// A^T A without explicitly forming A^T A").  For every row, the columns
// that contain it are linked through the most recent such column; union
// with path compression (Liu's algorithm).
void column_etree(const Pattern &P, std::vector<int32_t> &parent)
{
    const int32_t n = P.n;
    parent.assign(n, -1);
    std::vector<int32_t> anc(n, -1), prev(n, -1);
    for (int32_t k = 0; k < n; k++) {
        const int32_t c = P.Q[k];
        for (int32_t p = P.Ap[c]; p < P.Ap[c + 1]; p++) {
            int32_t i = prev[P.Ai[p]];
            while (i != -1 && i < k) {
                int32_t next = anc[i];
                anc[i] = k;
                if (next == -1) { parent[i] = k; break; }
                i = next;
            }
            prev[P.Ai[p]] = k;
        }
    }
}

// Levels of a dependency DAG given column-wise: dependencies of column k are
// the rows j < k of its U part.  Returns the number of levels.
int32_t levels_of(int32_t n, const int64_t *Up, const int32_t *Ui,
                  const int32_t *nU, std::vector<int32_t> &level, int32_t cut)
{
    level.assign(n, 0);
    int32_t nl = 0;
    for (int32_t k = 0; k < n; k++) {
        int32_t lv = 0;
        const int64_t end = nU ? Up[k] + nU[k] : Up[k + 1];
        for (int64_t e = Up[k]; e < end; e++) {
            const int32_t j = Ui[e];
            if (k >= cut && j >= cut) continue;
            if (j < k && level[j] + 1 > lv) lv = level[j] + 1;
        }
        level[k] = lv;
        if (lv + 1 > nl) nl = lv + 1;
    }
    return nl;
}

// EGraph levels of a Cholesky-pattern structure (symmetric_structure).
// Column k depends on the steps of its row subtree, which holds every child
// of k in the elimination tree (the parent of j is the first L row of
// column j), and each step depends on its own children, so levels grow up
// every tree path and the level of k is its height: one more than its
// highest child, 0 for a leaf.  Equals levels_of on such a structure.
static int32_t tree_levels(const Structure &S, std::vector<int32_t> &level)
{
    const int32_t n = S.n;
    level.assign(n, 0);
    int32_t nl = n > 0 ? 1 : 0;
    for (int32_t j = 0; j < n; j++) {
        const int64_t l0 = S.LUp[j] + S.nU[j];
        if (l0 >= S.LUp[j + 1]) continue;
        const int32_t p = S.LUi[l0];
        if (level[j] + 1 > level[p]) level[p] = level[j] + 1;
        if (level[p] + 1 > nl) nl = level[p] + 1;
    }
    return nl;
}

// Lower adjacency of S = (A + A^T)(Q,Q) by row (cnt[n+1] offsets; the steps j < i
// adjacent to step i) and the elimination tree of S (Liu's algorithm with
// path compression).
static void symmetric_graph(const Pattern &P, std::vector<int64_t> &cnt, std::vector<int32_t> &lowadj,
                            std::vector<int32_t> &parent, const int32_t *rowstep = nullptr)
{
    const int32_t n = P.n;
    // entry A(r, c) joins the steps rowstep[r] (qinv[r] by default) and qinv[c]
    const int32_t *rs = rowstep ? rowstep : P.qinv.data();
    cnt.assign(n + 1, 0);
    for (int32_t c = 0; c < n; c++)
        for (int32_t p = P.Ap[c]; p < P.Ap[c + 1]; p++) {
            const int32_t i = rs[P.Ai[p]], j = P.qinv[c];
            if (i != j) cnt[std::max(i, j) + 1]++;
        }
    for (int32_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    lowadj.assign(cnt[n], 0);
    {
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        for (int32_t c = 0; c < n; c++)
            for (int32_t p = P.Ap[c]; p < P.Ap[c + 1]; p++) {
                const int32_t i = rs[P.Ai[p]], j = P.qinv[c];
                if (i != j) lowadj[pos[std::max(i, j)]++] = std::min(i, j);
            }
    }
    std::vector<int32_t> anc(n, -1);
    parent.assign(n, -1);
    for (int32_t k = 0; k < n; k++) {
        for (int64_t e = cnt[k]; e < cnt[k + 1]; e++) {
            int32_t i = lowadj[e];
            while (i != -1 && i < k) {
                const int32_t next = anc[i];
                anc[i] = k;
                if (next == -1) parent[i] = k;
                i = next;
            }
        }
    }
}

// Number of entries of the strict lower Cholesky factor of
// S = (A + A^T)(Q,Q): row structures come from the elimination tree of S by
// walking up from every off-diagonal entry of row k until a node already
// visited for row k ("row subtree").  When every diagonal pivot is kept on a
// structurally symmetric matrix, L and U^T both have this pattern; it sizes
// the pool of the first factorization (pivoting can change it, and the pool
// then grows).  With c_j the entries of column j, the factorization then
// costs F = sum_j 2 c_j^2 flops (every U(j,k) != 0 uses the c_j entries of
// L(:,j), and U(j,:) has c_j entries above the diagonal): *flops.
int64_t symmetric_fill(const Pattern &P, double *flops)
{
    const int32_t n = P.n;
    std::vector<int64_t> cnt;
    std::vector<int32_t> lowadj, parent, mark(n, -1);
    symmetric_graph(P, cnt, lowadj, parent);
    int64_t total = 0;
    std::vector<int64_t> colcount(flops ? n : 0, 0);
    for (int32_t k = 0; k < n; k++) {
        mark[k] = k;
        for (int64_t e = cnt[k]; e < cnt[k + 1]; e++)
            for (int32_t j = lowadj[e]; j != -1 && mark[j] != k; j = parent[j]) {
                mark[j] = k;
                total++;
                if (flops) colcount[j]++;
            }
    }
    if (flops) {
        *flops = 0.0;
        for (int64_t c : colcount) *flops += 2.0 * (double)c * (double)c;
    }
    return total;
}

// Partition point and trapezoid slices of one triangular factor (Section
// V-A).  count_from[p] = entries of the trailing block [p, n) (suffix sums of
// the per-column (lower) or per-row (upper) strict counts); rowlen[i] = all
// entries of row i of the factor.  Paper's rule (density == 0): scan down
// from n-1 and stop at the first position whose trailing block holds at
// least frac * total and min_entries entries (the smallest such block).
// GPU rule (density > 0): P0 = the start of the longest trailing block whose
// entry density count_from[p] / ((n-p)(n-p-1)/2) is at least `density`,
// kept if it holds min_entries entries.  The rows [P0, n) are cut into
// `slices` pieces of equal entry counts (at most max_piece rows each).
// Returns n when no block qualifies.
// fn(k0, k1, t) on up to kHostThreads host threads t over index ranges
// [k0, k1) of about equal weight (ptr: n+1 ascending offsets, the weight of
// index k is ptr[k+1] - ptr[k]); small inputs run on the calling thread
constexpr int kHostThreads = 16;

template <class T, class F>
static void parallel_ranges(int32_t n, const T *ptr, F &&fn)
{
    const int nt = (int)std::max(1u, std::min((unsigned)kHostThreads, std::thread::hardware_concurrency()));
    const int64_t total = n > 0 ? (int64_t)ptr[n] - (int64_t)ptr[0] : 0;
    if (nt == 1 || total < (1 << 20)) {
        fn(0, n, 0);
        return;
    }
    std::vector<std::thread> th;
    int32_t k0 = 0;
    for (int t = 1; t <= nt; t++) {
        int32_t k1 = n;
        if (t < nt) {
            const T target = (T)((int64_t)ptr[0] + total * t / nt);
            k1 = (int32_t)(std::lower_bound(ptr, ptr + n + 1, target) - ptr);
        }
        k1 = std::min(std::max(k1, k0), n);
        if (k1 > k0) th.emplace_back(fn, k0, k1, t - 1);
        k0 = k1;
    }
    for (std::thread &x : th) x.join();
}

// fn(k0, k1, t) over chunks [k0, k1) of `chunk` indices, taken in turn by
// up to kHostThreads host threads t as each finishes its previous chunk (for
// work whose cost per index is not known in advance)
template <class F>
static void parallel_chunks(int32_t n, int32_t chunk, F &&fn)
{
    const int nt = (int)std::max(1u, std::min((unsigned)kHostThreads, std::thread::hardware_concurrency()));
    if (nt == 1 || n <= chunk) {
        if (n > 0) fn(0, n, 0);
        return;
    }
    std::atomic<int64_t> next{0};
    auto run = [&](int t) {
        for (;;) {
            const int64_t k0 = next.fetch_add(chunk);
            if (k0 >= n) break;
            fn((int32_t)k0, (int32_t)std::min<int64_t>(n, k0 + chunk), t);
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; t++) th.emplace_back(run, t);
    run(0);
    for (std::thread &x : th) x.join();
}

static int32_t dense_split(int32_t n, const std::vector<int64_t> &count_from, const std::vector<int64_t> &rowlen,
                           const SolveSplit &sp, std::vector<int32_t> &cut)
{
    cut.clear();
    const int64_t total = count_from.empty() ? 0 : count_from[0];
    if (sp.slices <= 0 || total <= 0) return n;
    int32_t p0 = n;
    if (sp.density > 0.0) {
        for (int32_t p = n - 2; p >= 0; p--) {
            const double m = (double)(n - p);
            if ((double)count_from[p] < sp.density * m * (m - 1.0) / 2.0) break;
            p0 = p;
        }
        if (p0 < n && count_from[p0] < sp.min_entries) p0 = n;
    } else {
        for (int32_t p = n - 1; p >= 0; p--) {
            if ((double)count_from[p] >= sp.frac * (double)total && count_from[p] >= sp.min_entries) {
                p0 = p;
                break;
            }
        }
    }
    if (p0 >= n) return n;
    int64_t tot = 0;
    for (int32_t i = p0; i < n; i++) tot += rowlen[i];
    const double per = (double)tot / sp.slices;
    cut.push_back(p0);
    int64_t acc = 0;
    int32_t start = p0;
    for (int32_t i = p0; i < n; i++) {
        acc += rowlen[i];
        if (i + 1 < n && ((double)acc >= per || i + 1 - start >= sp.max_piece)) {
            cut.push_back(i + 1);
            acc = 0;
            start = i + 1;
        }
    }
    cut.push_back(n);
    return p0;
}

// Row-wise (CSR) copies of L and U for the solves and the wide columns:
// per-thread histograms of the row entries over column ranges give each
// range its first position in every row; each thread then copies its
// columns in ascending order, so every row lists its entries by ascending
// column, as a serial pass would.
static void rowwise_copies(const Structure &S, Schedule &W)
{
    const int32_t n = S.n;
    W.Lrp.assign(n + 1, 0);
    W.Urp.assign(n + 1, 0);
    W.Udiag.assign(n, 0);
    {
        std::vector<std::vector<int64_t>> hl(kHostThreads), hu(kHostThreads);
        parallel_ranges(n, S.LUp.data(), [&](int32_t k0, int32_t k1, int t) {
            std::vector<int64_t> &cl = hl[t], &cu = hu[t];
            cl.assign(n, 0);
            cu.assign(n, 0);
            for (int32_t k = k0; k < k1; k++) {
                const int64_t d = S.LUp[k] + S.nU[k] - 1;
                W.Udiag[k] = (int32_t)d;
                for (int64_t e = S.LUp[k]; e < d; e++) cu[S.LUi[e]]++;
                for (int64_t e = d + 1; e < S.LUp[k + 1]; e++) cl[S.LUi[e]]++;
            }
        });
        for (int t = 0; t < kHostThreads; t++) {
            if (hl[t].empty()) continue;
            for (int32_t i = 0; i < n; i++) {
                W.Lrp[i + 1] += hl[t][i];
                W.Urp[i + 1] += hu[t][i];
            }
        }
        for (int32_t i = 0; i < n; i++) {
            W.Lrp[i + 1] += W.Lrp[i];
            W.Urp[i + 1] += W.Urp[i];
        }
        std::vector<int64_t> lp(W.Lrp.begin(), W.Lrp.end() - 1), up(W.Urp.begin(), W.Urp.end() - 1);
        for (int t = 0; t < kHostThreads; t++) {
            if (hl[t].empty()) continue;
            for (int32_t i = 0; i < n; i++) {
                const int64_t a = hl[t][i], b = hu[t][i];
                hl[t][i] = lp[i];
                hu[t][i] = up[i];
                lp[i] += a;
                up[i] += b;
            }
        }
        W.Lcol.resize(W.Lrp[n]);
        W.Lslot.resize(W.Lrp[n]);
        W.Urow_col.resize(W.Urp[n]);
        W.Uslot.resize(W.Urp[n]);
        parallel_ranges(n, S.LUp.data(), [&](int32_t k0, int32_t k1, int t) {
            std::vector<int64_t> &ol = hl[t], &ou = hu[t];
            for (int32_t k = k0; k < k1; k++) {
                const int64_t d = S.LUp[k] + S.nU[k] - 1;
                for (int64_t e = S.LUp[k]; e < d; e++) {
                    const int64_t q = ou[S.LUi[e]]++;
                    W.Urow_col[q] = k;
                    W.Uslot[q] = (int32_t)e;
                }
                for (int64_t e = d + 1; e < S.LUp[k + 1]; e++) {
                    const int64_t q = ol[S.LUi[e]]++;
                    W.Lcol[q] = k;
                    W.Lslot[q] = (int32_t)e;
                }
            }
        });
    }
    W.rowwise_ready = true;
}

// The solve part of the schedule (Section V and the row blocks of the
// sparse solves), which the re-factorization does not read: the original
// row ids of the restart kernel, the row-wise copies (unless the wide
// columns needed them already), the structure-adaptive split, the
// trailing block's slices and the row blocks with their levels.
void build_solve_schedule(const Structure &S, const SolveSplit &split, Schedule &W)
{
    const int32_t n = S.n;
    const double thr = W.thr;
    // ---- original row ids of L entries (used by the restart kernel) ----
    W.LUi_orig.resize(S.LUi.size());
    parallel_ranges(n, S.LUp.data(), [&](int32_t k0, int32_t k1, int) {
        for (int32_t k = k0; k < k1; k++)
            for (int64_t e = S.LUp[k]; e < S.LUp[k + 1]; e++)
                W.LUi_orig[e] = (e - S.LUp[k] >= S.nU[k]) ? S.piv[S.LUi[e]] : S.LUi[e];
    });
    if (!W.rowwise_ready) rowwise_copies(S, W);
    // ---- structure-adaptive split of both triangular factors (Section V) ----
    {
        std::vector<int64_t> cf(n + 1, 0), rl(n, 0);
        for (int32_t j = n - 1; j >= 0; j--)
            cf[j] = cf[j + 1] + (S.LUp[j + 1] - S.LUp[j] - S.nU[j]);
        for (int32_t i = 0; i < n; i++) rl[i] = W.Lrp[i + 1] - W.Lrp[i];
        W.lp0 = dense_split(n, cf, rl, split, W.lcut);
        std::vector<int64_t> cu(n + 1, 0), ru(n, 0);
        for (int32_t i = n - 1; i >= 0; i--) cu[i] = cu[i + 1] + (W.Urp[i + 1] - W.Urp[i]);
        for (int32_t i = 0; i < n; i++) ru[i] = W.Urp[i + 1] - W.Urp[i];
        W.up0 = dense_split(n, cu, ru, split, W.ucut);
    }
    // ---- row blocks of the sparse solves and their levels ----
    // forward: rows i-1 and i share a block when L(:,i-1) = {i} + L(:,i)
    // (then row f+q holds L(f+q, f..f+q-1) as its last q entries);
    // backward: when U(i-1,:) = {i} + U(i,:) off the diagonal (then row f+q
    // holds U(f+q, f+q+1..l-1) as its first l-1-f-q entries)
    auto blocks = [&](int32_t nrows, bool lower, std::vector<int32_t> &bs) {
        bs.assign(1, 0);
        for (int32_t i = 1; i < nrows; i++) {
            bool link;
            if (lower) {
                link = W.chain[i - 1] != 0;
            } else {
                const int64_t a0 = W.Urp[i - 1], a1 = W.Urp[i], b1 = W.Urp[i + 1];
                link = (a1 - a0 == b1 - a1 + 1) && W.Urow_col[a0] == i &&
                       std::equal(W.Urow_col.begin() + a0 + 1, W.Urow_col.begin() + a1, W.Urow_col.begin() + a1);
            }
            if (!link || i - bs.back() >= kSolveBlockRows) bs.push_back(i);
        }
        if (nrows > 0) bs.push_back(nrows);
    };
    blocks(W.lp0, true, W.lbs);
    blocks(W.up0, false, W.ubs);
    // levels of the blocks: forward over ascending blocks, backward over
    // descending ones; a block waits for the blocks of its rows' entries
    // outside it (entries in the dense part are final before)
    auto levelize = [&](bool lower, const std::vector<int32_t> &bs, std::vector<int32_t> &ptr,
                        std::vector<int32_t> &ids, std::vector<int32_t> &tptr, std::vector<int32_t> &tick,
                        std::vector<int32_t> &rbk, int32_t &nlev, int32_t &div) {
        const int32_t nb = bs.empty() ? 0 : (int32_t)bs.size() - 1;
        const int32_t nrows = nb ? bs[nb] : 0;
        std::vector<int32_t> blk(nrows), lv(nb, 0);
        for (int32_t b = 0; b < nb; b++)
            for (int32_t i = bs[b]; i < bs[b + 1]; i++) blk[i] = b;
        nlev = 0;
        for (int32_t t = 0; t < nb; t++) {
            const int32_t b = lower ? t : nb - 1 - t;
            int32_t v = 0;
            for (int32_t i = bs[b]; i < bs[b + 1]; i++) {
                const std::vector<int64_t> &rp = lower ? W.Lrp : W.Urp;
                const BigVec<int32_t> &cc = lower ? W.Lcol : W.Urow_col;
                for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
                    const int32_t j = cc[e];
                    if (j < nrows && blk[j] != b) v = std::max(v, lv[blk[j]] + 1);
                }
            }
            lv[b] = v;
            nlev = std::max(nlev, v + 1);
        }
        ptr.assign(nlev + 1, 0);
        for (int32_t b = 0; b < nb; b++) ptr[lv[b] + 1]++;
        for (int32_t l = 0; l < nlev; l++) ptr[l + 1] += ptr[l];
        ids.assign(nb, 0);
        std::vector<int32_t> pos(ptr.begin(), ptr.end() - 1);
        for (int32_t t = 0; t < nb; t++) {
            const int32_t b = lower ? t : nb - 1 - t;
            ids[pos[lv[b]]++] = b;
        }
        tptr.assign(nlev + 1, 0);
        tick.clear();
        tick.reserve(nrows);
        for (int32_t l = 0; l < nlev; l++) {
            for (int32_t p = ptr[l]; p < ptr[l + 1]; p++) {
                const int32_t b = ids[p];
                if (lower)
                    for (int32_t i = bs[b]; i < bs[b + 1]; i++) tick.push_back(i);
                else
                    for (int32_t i = bs[b + 1] - 1; i >= bs[b]; i--) tick.push_back(i);
            }
            tptr[l + 1] = (int32_t)tick.size();
        }
        rbk = blk;
        // a level is run as its own launches while it has at least as many
        // rows as the threshold
        div = nlev;
        for (int32_t l = 0; l < nlev; l++)
            if ((double)(tptr[l + 1] - tptr[l]) < thr) { div = l; break; }
    };
    // the two triangles' levels are independent, and independent of the
    // trailing block's slices below
    std::thread upper([&]() {
        levelize(false, W.ubs, W.usv_ptr, W.usv_rows, W.usv_tptr, W.usv_tick, W.urb, W.usv_levels, W.usv_div);
    });
    std::thread lower([&]() {
        levelize(true, W.lbs, W.lsv_ptr, W.lsv_rows, W.lsv_tptr, W.lsv_tick, W.lrb, W.lsv_levels, W.lsv_div);
    });
    // ---- trailing block in 32-row slices (forward L, backward U), over
    // column chunks on the host threads; a column's rows ascend, so the
    // slice boundaries are found in one walk down them ----
    W.ltri0.clear();
    W.lseg.clear();
    W.lnb = 0;
    if (W.lp0 < n) {
        const int32_t m = n - W.lp0, nb = (m + kTrailRows - 1) / kTrailRows;
        W.lnb = nb;
        W.ltri0.resize(m);
        W.lseg.resize((size_t)m * (nb + 1));
        parallel_chunks(m, 256, [&](int32_t a, int32_t b, int) {
            for (int32_t i = W.lp0 + a; i < W.lp0 + b; i++) {
                const int32_t *c = W.Lcol.data() + W.Lrp[i];
                const int32_t len = (int32_t)(W.Lrp[i + 1] - W.Lrp[i]);
                W.ltri0[i - W.lp0] = W.Lrp[i] + (std::lower_bound(c, c + len, W.lp0) - c);
            }
            for (int32_t j = W.lp0 + a; j < W.lp0 + b; j++) {
                const int32_t *r = S.LUi.data() + S.LUp[j] + S.nU[j];
                const int32_t len = (int32_t)(S.LUp[j + 1] - S.LUp[j] - S.nU[j]);
                int32_t *sg = W.lseg.data() + (size_t)(j - W.lp0) * (nb + 1);
                int32_t pos = 0;
                for (int32_t I = 0; I <= nb; I++) {
                    const int64_t lo = (int64_t)W.lp0 + (int64_t)kTrailRows * I;
                    if (lo >= n) {
                        sg[I] = len;
                        continue;
                    }
                    while (pos < len && r[pos] < lo) pos++;
                    sg[I] = pos;
                }
            }
        });
    }
    W.ufar.clear();
    W.useg.clear();
    W.unb = 0;
    if (W.up0 < n) {
        const int32_t m = n - W.up0, nb = (m + kTrailRows - 1) / kTrailRows;
        W.unb = nb;
        W.ufar.resize(W.up0);
        parallel_chunks(W.up0, 2048, [&](int32_t a, int32_t b, int) {
            for (int32_t i = a; i < b; i++) {
                const int32_t *c = W.Urow_col.data() + W.Urp[i];
                const int32_t len = (int32_t)(W.Urp[i + 1] - W.Urp[i]);
                W.ufar[i] = W.Urp[i] + (std::lower_bound(c, c + len, W.up0) - c);
            }
        });
        W.useg.resize((size_t)m * (nb + 1));
        parallel_chunks(m, 256, [&](int32_t a, int32_t b, int) {
            for (int32_t j = W.up0 + a; j < W.up0 + b; j++) {
                const int32_t *r = S.LUi.data() + S.LUp[j];
                const int32_t len = S.nU[j];   // U rows ascending, the diagonal (row j) last
                int32_t *sg = W.useg.data() + (size_t)(j - W.up0) * (nb + 1);
                int32_t pos = 0;
                for (int32_t I = 0; I <= nb; I++) {
                    const int64_t lo = (int64_t)W.up0 + (int64_t)kTrailRows * I;
                    if (lo >= n) {
                        sg[I] = len;
                        continue;
                    }
                    while (pos < len && r[pos] < lo) pos++;
                    sg[I] = pos;
                }
            }
        });
    }
    lower.join();
    upper.join();
    W.solve_ready = true;
}

void build_schedule(const Pattern &P, const Structure &S, double alpha,
                    int resident_warps, int sched_mode, int cap_short, const SolveSplit &split,
                    int dense_min_rows, Schedule &W, bool defer_solve)
{
    const int32_t n = S.n;
    W.rowwise_ready = false;
    W.solve_ready = false;
    // ---- dense tail: the longest trailing block [p, n) in which every
    // column holds every row >= p (low[k] = first row of the unbroken run of
    // rows that ends at n-1 in column k) ----
    W.dense_p = n;
    W.dense_m = 0;
    W.dense_s0.clear();
    if (dense_min_rows > 0 && n > 0) {
        int32_t pd = n, mx = 0;
        for (int32_t p = n - 1; p >= 0; p--) {
            const int64_t b = S.LUp[p], e = S.LUp[p + 1];
            int32_t low = n;
            if (e > b && S.LUi[e - 1] == n - 1) {
                int64_t q = e - 1;
                while (q > b && S.LUi[q - 1] == S.LUi[q] - 1) q--;
                low = S.LUi[q];
            }
            mx = std::max(mx, low);
            if (mx > p) break;
            pd = p;
        }
        int32_t m = n - pd;
        if (m > GBLU_DENSE_MAX_ROWS) { m = GBLU_DENSE_MAX_ROWS; pd = n - m; }
        if (m >= dense_min_rows) {
            W.dense_p = pd;
            W.dense_m = m;
            W.dense_s0.resize(m);
            for (int32_t c = 0; c < m; c++) {
                const int32_t k = pd + c;
                const int32_t *r = S.LUi.data() + S.LUp[k];
                const int32_t len = (int32_t)(S.LUp[k + 1] - S.LUp[k]);
                W.dense_s0[c] = (int32_t)(std::lower_bound(r, r + len, pd) - r);
            }
        }
    }
    // ---- supernode links of L: L(:,j) = {j+1} + L(:,j+1) ----
    W.chain.assign(n, 0);
    parallel_ranges(n, S.LUp.data(), [&](int32_t j0, int32_t j1, int) {
        for (int32_t j = j0; j < j1 && j + 1 < n; j++) {
            const int64_t a = S.LUp[j] + S.nU[j], ae = S.LUp[j + 1];
            const int64_t b = S.LUp[j + 1] + S.nU[j + 1], be = S.LUp[j + 2];
            if (ae - a != be - b + 1 || S.LUi[a] != j + 1) continue;
            W.chain[j] = std::equal(S.LUi.begin() + a + 1, S.LUi.begin() + ae, S.LUi.begin() + b) ? 1 : 0;
        }
    });
    // ---- wide columns: at most kPullMaxL L entries and at least kPullMinRuns
    // supernode runs among the dependencies.  All but the last chain of linked
    // dependencies are taken row by row (pull_start = where that chain
    // starts); none in the dense tail ----
    W.pull_start.assign(n, 0);
    {
        std::atomic<int64_t> cnt{0};
        parallel_ranges(n, S.LUp.data(), [&](int32_t k0, int32_t k1, int) {
            int64_t c = 0;
            for (int32_t k = k0; k < k1 && k < W.dense_p; k++) {
                const int64_t b = S.LUp[k];
                const int32_t nd = S.nU[k] - 1, nl = (int32_t)(S.LUp[k + 1] - b) - S.nU[k];
                if (nl > kPullMaxL || nd < kPullMinRuns) continue;
                const int32_t *u = S.LUi.data() + b;
                auto linked = [&](int32_t i) { return u[i] == u[i - 1] + 1 && W.chain[u[i - 1]] != 0; };
                int32_t runs = 1;
                for (int32_t i = 1; i < nd; i++) runs += !linked(i);
                if (runs < kPullMinRuns) continue;
                int32_t p = nd - 1;
                while (p > 0 && linked(p)) p--;
                W.pull_start[k] = p;
                c += p > 0;
            }
            cnt += c;
        });
        W.pull_cols = cnt.load();
    }
    const double thr = alpha * (double)resident_warps;
    W.thr = thr;
    // ---- EGraph levels, the dividing level (Section IV-B) and the tasks:
    // on a thread of their own, beside the slot maps and row-wise copies
    // below (they write disjoint members of W) ----
    std::thread level_thread([&]() {
        // columns of the dense tail wait only for their dependencies before it
        std::vector<int32_t> level;
        W.n_levels = S.symmetric && W.dense_p >= n ? tree_levels(S, level)
                                                   : levels_of(n, S.LUp.data(), S.LUi.data(), S.nU.data(), level,
                                                               W.dense_p);
        W.level_ptr.assign(W.n_levels + 1, 0);
        for (int32_t k = 0; k < n; k++) W.level_ptr[level[k] + 1]++;
        for (int32_t l = 0; l < W.n_levels; l++) W.level_ptr[l + 1] += W.level_ptr[l];
        W.level_cols.assign(n, 0);
        {
            std::vector<int32_t> pos(W.level_ptr.begin(), W.level_ptr.end() - 1);
            for (int32_t k = 0; k < n; k++) W.level_cols[pos[level[k]]++] = k;
        }
        W.div_level = W.n_levels;
        for (int32_t l = 0; l < W.n_levels; l++)
            if ((double)(W.level_ptr[l + 1] - W.level_ptr[l]) < thr) { W.div_level = l; break; }
        if (sched_mode == GBLU_SCHED_LEVEL) W.div_level = W.n_levels;
        if (sched_mode == GBLU_SCHED_SYNCFREE) W.div_level = 0;
        // ---- tasks, in level order: long columns alone, medium columns in pairs,
        // short ones in groups of up to 8.  A pending item is only merged with
        // the column that immediately follows it, so a task never comes before
        // a task holding one of its dependencies.  Groups stay inside a level
        // before the dividing level.
        W.task_ptr.assign(1, 0);
        W.task_cols.clear();
        W.task_cols.reserve(n);
        W.level_task_ptr.assign(1, 0);
        {
            const int64_t half = kRefCapLong / 2;   // medium: up to half the CTA's entries
            int32_t group = 0;      // short columns pending
            bool pend_med = false;  // one medium column pending
            auto close = [&]() {
                if (group || pend_med) W.task_ptr.push_back((int32_t)W.task_cols.size());
                group = 0;
                pend_med = false;
            };
            for (int32_t l = 0; l < W.n_levels; l++) {
                for (int32_t p = W.level_ptr[l]; p < W.level_ptr[l + 1]; p++) {
                    const int32_t k = W.level_cols[p];
                    const int64_t len = S.LUp[k + 1] - S.LUp[k];
                    if (len > half || W.pull_start[k] > 0) {   // a whole CTA
                        close();
                        W.task_cols.push_back(k);
                        W.task_ptr.push_back((int32_t)W.task_cols.size());
                    } else if (len > cap_short) {
                        if (pend_med) {
                            W.task_cols.push_back(k);
                            W.task_ptr.push_back((int32_t)W.task_cols.size());
                            pend_med = false;
                        } else {
                            close();
                            W.task_cols.push_back(k);
                            pend_med = true;
                        }
                    } else {
                        if (pend_med) close();
                        W.task_cols.push_back(k);
                        if (++group == 8) close();
                    }
                }
                if (l < W.div_level) {
                    close();
                    W.level_task_ptr.push_back((int32_t)W.task_ptr.size() - 1);
                }
            }
            close();
        }
    });
    // ---- flops of one refactorization (partial sums of integers, exact in
    // any order below 2^53) ----
    double part[kHostThreads] = {};
    parallel_ranges(n, S.LUp.data(), [&](int32_t k0, int32_t k1, int t) {
        double fl = 0;
        for (int32_t k = k0; k < k1; k++)
            for (int64_t e = S.LUp[k]; e < S.LUp[k] + S.nU[k] - 1; e++) {
                const int32_t j = S.LUi[e];
                fl += 2.0 * (double)(S.LUp[j + 1] - S.LUp[j] - S.nU[j]);
            }
        part[t] = fl;
    });
    W.flops = 0;
    for (double v : part) W.flops += v;
    // ---- A slot -> position in its column (columns are sorted) ----
    const int64_t nnzA = (int64_t)P.Ai.size();
    W.amap.assign(nnzA, -1);
    parallel_chunks(n, 2048, [&](int32_t c0, int32_t c1, int) {
        for (int32_t c = c0; c < c1; c++) {
            const int32_t k = P.qinv[c];
            const int32_t *col = S.LUi.data() + S.LUp[k];
            const int32_t len = (int32_t)(S.LUp[k + 1] - S.LUp[k]);
            for (int32_t p = P.Ap[c]; p < P.Ap[c + 1]; p++) {
                const int32_t s = S.pinv[P.Ai[p]];
                const int32_t *it = std::lower_bound(col, col + len, s);
                W.amap[p] = (it != col + len && *it == s) ? (int32_t)(it - col) : -1;
            }
        }
    });
    if (defer_solve) {
        // the wide columns read rows of L during the re-factorization
        if (W.pull_cols > 0) rowwise_copies(S, W);
        level_thread.join();
        return;
    }
    build_solve_schedule(S, split, W);
    level_thread.join();
}

// Off-diagonal entries of A whose transposed position is not an entry of A
// (duplicates counted once per entry); A is structurally symmetric at 0.
int64_t unsymmetric_entries(const Pattern &P)
{
    const int32_t n = P.n;
    std::vector<int32_t> rp(n + 1, 0);
    for (int32_t p = 0; p < P.Ap[n]; p++) rp[P.Ai[p] + 1]++;
    for (int32_t i = 0; i < n; i++) rp[i + 1] += rp[i];
    std::vector<int32_t> cols(P.Ap[n]);
    {
        std::vector<int32_t> pos(rp.begin(), rp.end() - 1);
        for (int32_t c = 0; c < n; c++)
            for (int32_t p = P.Ap[c]; p < P.Ap[c + 1]; p++) cols[pos[P.Ai[p]]++] = c;
    }
    // column j's rows marked; row j's columns c must each be marked (A(c, j))
    std::vector<int32_t> mark(n, -1);
    int64_t miss = 0;
    for (int32_t j = 0; j < n; j++) {
        for (int32_t p = P.Ap[j]; p < P.Ap[j + 1]; p++) mark[P.Ai[p]] = j;
        for (int32_t e = rp[j]; e < rp[j + 1]; e++) miss += cols[e] != j && mark[cols[e]] != j;
    }
    return miss;
}

// Factor structure of a first factorization that predicts every step to
// keep its diagonal row (piv = Q; or the rows piv[k] when given, with A
// read as B = A(piv, Q) below).  L and U^T take the pattern of the
// Cholesky factor of S = (A + A^T)(Q,Q): column k holds the row subtree of k
// in the elimination tree of S (its U rows, ascending), k itself, then the
// rows i > k whose row subtree contains k.  This pattern contains the
// pattern of the LU factors of A(Q,Q) without row exchanges, and equals it
// when A is structurally symmetric (George and Ng); an entry outside the
// exact pattern only sums products with a structural zero, so it computes to
// an exact zero for finite values.  Three passes over the row subtrees on
// host threads: their sizes, then over fixed row ranges the L entries each
// range gives every column, then the entries themselves, each range writing
// its own part of every L column so that the rows stay ascending.
void symmetric_structure(const Pattern &P, Structure &S, const std::vector<int32_t> *piv)
{
    const int32_t n = P.n;
    std::vector<int32_t> pinv;
    if (piv) {
        pinv.assign(n, -1);
        for (int32_t k = 0; k < n; k++) pinv[(*piv)[k]] = k;
    }
    std::vector<int64_t> adjp;
    std::vector<int32_t> adj, parent;
    symmetric_graph(P, adjp, adj, parent, piv ? pinv.data() : nullptr);
    // walk(k, fn): fn(j) for every j of the row subtree of k
    auto walk = [&](int32_t k, std::vector<int32_t> &mark, auto &&fn) {
        mark[k] = k;
        for (int64_t e = adjp[k]; e < adjp[k + 1]; e++)
            for (int32_t j = adj[e]; mark[j] != k; j = parent[j]) {
                mark[j] = k;
                fn(j);
            }
    };
    std::vector<int64_t> rowp(n + 1, 0);
    {
        std::vector<std::vector<int32_t>> marks(kHostThreads);
        parallel_chunks(n, 1024, [&](int32_t k0, int32_t k1, int t) {
            std::vector<int32_t> &mark = marks[t];
            if (mark.empty()) mark.assign(n, -1);
            for (int32_t k = k0; k < k1; k++) {
                int64_t c = 0;
                walk(k, mark, [&](int32_t) { c++; });
                rowp[k + 1] = c;
            }
        });
    }
    for (int32_t k = 0; k < n; k++) rowp[k + 1] += rowp[k];
    std::vector<std::vector<int32_t>> part(kHostThreads);
    parallel_ranges(n, rowp.data(), [&](int32_t k0, int32_t k1, int t) {
        std::vector<int32_t> mark(n, -1);
        std::vector<int32_t> &c = part[t];
        c.assign(n, 0);
        for (int32_t k = k0; k < k1; k++) walk(k, mark, [&](int32_t j) { c[j]++; });
    });
    S.n = n;
    S.LUp.assign(n + 1, 0);
    S.nU.assign(n, 0);
    for (int32_t k = 0; k < n; k++) {
        int64_t nl = 0;
        for (const std::vector<int32_t> &c : part)
            if (!c.empty()) nl += c[k];
        S.nU[k] = (int32_t)(rowp[k + 1] - rowp[k]) + 1;
        S.LUp[k + 1] = S.LUp[k] + S.nU[k] + nl;
    }
    // each range's first slot in every L column, ranges in ascending order
    for (int32_t k = 0; k < n; k++) {
        int64_t o = S.LUp[k] + S.nU[k];
        for (std::vector<int32_t> &c : part)
            if (!c.empty()) {
                const int32_t m = c[k];
                c[k] = (int32_t)(o - S.LUp[k]);
                o += m;
            }
    }
    S.LUi.resize(S.LUp[n]);
    int32_t *LUi = S.LUi.data();
    // the walk from one entry of row k climbs the tree to ascending steps, so
    // the U rows of column k come as ascending runs, merged pairwise
    parallel_ranges(n, rowp.data(), [&](int32_t k0, int32_t k1, int t) {
        std::vector<int32_t> mark(n, -1), bnd, tmp;
        std::vector<int32_t> &off = part[t];
        for (int32_t k = k0; k < k1; k++) {
            int32_t *u = LUi + S.LUp[k];
            int32_t m = 0;
            bnd.clear();
            mark[k] = k;
            for (int64_t e = adjp[k]; e < adjp[k + 1]; e++) {
                int32_t j = adj[e];
                if (mark[j] == k) continue;
                bnd.push_back(m);
                for (; mark[j] != k; j = parent[j]) {
                    mark[j] = k;
                    u[m++] = j;
                    LUi[S.LUp[j] + off[j]++] = k;
                }
            }
            size_t nr = bnd.size();
            bnd.push_back(m);
            if (nr > 1) {
                tmp.resize(m);
                int32_t *src = u, *dst = tmp.data();
                while (nr > 1) {
                    size_t w = 0;
                    for (size_t r = 0; r < nr; r += 2) {
                        const int32_t a = bnd[r], mid = bnd[std::min(r + 1, nr)], b = bnd[std::min(r + 2, nr)];
                        std::merge(src + a, src + mid, src + mid, src + b, dst + a);
                        bnd[w++] = a;
                    }
                    bnd[w] = m;
                    nr = w;
                    std::swap(src, dst);
                }
                if (src != u) std::copy(src, src + m, u);
            }
            u[m] = k;
        }
    });
    if (piv) {
        S.piv = *piv;
        S.pinv = std::move(pinv);
    } else {
        S.piv = P.Q;
        S.pinv = P.qinv;
    }
    S.symmetric = true;
}

}  // namespace gblu


// ------------------------------------------------------------ host-only C ABI
using namespace gblu;

extern "C" int gblu_column_etree(int32_t n, const int32_t *Ap, const int32_t *Ai,
                                 const int32_t *Q, int32_t *parent)
{
    std::string err;
    if (validate_pattern(n, Ap, Ai, err) != GBLU_OK || !parent) return GBLU_ERR_INVALID_INPUT;
    Pattern P;
    P.n = n;
    P.Ap.assign(Ap, Ap + n + 1);
    P.Ai.assign(Ai, Ai + Ap[n]);
    P.Q.resize(n);
    std::vector<int32_t> seen(n, 0);
    for (int32_t k = 0; k < n; k++) {
        int32_t c = Q ? Q[k] : k;
        if (c < 0 || c >= n || seen[c]) return GBLU_ERR_INVALID_INPUT;
        seen[c] = 1;
        P.Q[k] = c;
    }
    std::vector<int32_t> par;
    column_etree(P, par);
    std::memcpy(parent, par.data(), sizeof(int32_t) * n);
    return GBLU_OK;
}

extern "C" int64_t gblu_restart_set(int32_t n, const int32_t *parent, const uint8_t *finished,
                                    uint8_t *out)
{
    if (n < 1 || !parent || !finished || !out) return GBLU_ERR_INVALID_INPUT;
    std::memset(out, 0, (size_t)n);
    int64_t cnt = 0;
    // Section IV-C: every unfinished node and all of its ancestors
    for (int32_t k = 0; k < n; k++) {
        if (finished[k]) continue;
        for (int32_t j = k; j != -1 && !out[j]; j = parent[j]) {
            out[j] = 1;
            cnt++;
        }
    }
    return cnt;
}

extern "C" int32_t gblu_levels(int32_t n, const int64_t *Up, const int32_t *Ui, int32_t *level)
{
    if (n < 1 || !Up || !Ui || !level) return GBLU_ERR_INVALID_INPUT;
    std::vector<int32_t> lv;
    int32_t nl = levels_of(n, Up, Ui, nullptr, lv);
    std::memcpy(level, lv.data(), sizeof(int32_t) * n);
    return nl;
}

extern "C" int gblu_symmetric_cost(int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *Q,
                                   int64_t *fill, double *flops)
{
    std::string err;
    if (validate_pattern(n, Ap, Ai, err) != GBLU_OK || !Q)
        return record_error(GBLU_ERR_INVALID_INPUT, "symmetric cost: invalid pattern or null Q");
    Pattern P;
    P.n = n;
    P.Ap.assign(Ap, Ap + n + 1);
    P.Ai.assign(Ai, Ai + Ap[n]);
    P.Q.assign(Q, Q + n);
    P.qinv.assign(n, -1);
    for (int32_t k = 0; k < n; k++) {
        if (Q[k] < 0 || Q[k] >= n || P.qinv[Q[k]] >= 0)
            return record_error(GBLU_ERR_INVALID_INPUT, "symmetric cost: Q is not a permutation");
        P.qinv[Q[k]] = k;
    }
    const int64_t f = symmetric_fill(P, flops);
    if (fill) *fill = f;
    return GBLU_OK;
}

extern "C" int64_t gblu_symmetric_structure(int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *Q,
                                            int64_t *LUp, int32_t *LUi, int32_t *nU)
{
    std::string err;
    if (validate_pattern(n, Ap, Ai, err) != GBLU_OK || !Q)
        return record_error(GBLU_ERR_INVALID_INPUT, "symmetric structure: invalid pattern or null Q");
    Pattern P;
    P.n = n;
    P.Ap.assign(Ap, Ap + n + 1);
    P.Ai.assign(Ai, Ai + Ap[n]);
    P.Q.assign(Q, Q + n);
    P.qinv.assign(n, -1);
    for (int32_t k = 0; k < n; k++) {
        if (Q[k] < 0 || Q[k] >= n || P.qinv[Q[k]] >= 0)
            return record_error(GBLU_ERR_INVALID_INPUT, "symmetric structure: Q is not a permutation");
        P.qinv[Q[k]] = k;
    }
    Structure S;
    symmetric_structure(P, S);
    if (LUp && LUi && nU) {
        std::memcpy(LUp, S.LUp.data(), sizeof(int64_t) * (n + 1));
        std::memcpy(nU, S.nU.data(), sizeof(int32_t) * n);
        std::memcpy(LUi, S.LUi.data(), sizeof(int32_t) * S.LUi.size());
    }
    return S.nnz();
}

extern "C" int64_t gblu_predicted_structure(int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *Q,
                                            const int32_t *piv, int64_t *LUp, int32_t *LUi, int32_t *nU)
{
    if (!piv) return gblu_symmetric_structure(n, Ap, Ai, Q, LUp, LUi, nU);
    std::string err;
    if (validate_pattern(n, Ap, Ai, err) != GBLU_OK || !Q)
        return record_error(GBLU_ERR_INVALID_INPUT, "predicted structure: invalid pattern or null Q");
    Pattern P;
    P.n = n;
    P.Ap.assign(Ap, Ap + n + 1);
    P.Ai.assign(Ai, Ai + Ap[n]);
    P.Q.assign(Q, Q + n);
    P.qinv.assign(n, -1);
    std::vector<int32_t> pv(piv, piv + n), seen(n, 0);
    for (int32_t k = 0; k < n; k++) {
        if (Q[k] < 0 || Q[k] >= n || P.qinv[Q[k]] >= 0 || pv[k] < 0 || pv[k] >= n || seen[pv[k]])
            return record_error(GBLU_ERR_INVALID_INPUT, "predicted structure: Q or piv is not a permutation");
        P.qinv[Q[k]] = k;
        seen[pv[k]] = 1;
    }
    Structure S;
    symmetric_structure(P, S, &pv);
    if (LUp && LUi && nU) {
        std::memcpy(LUp, S.LUp.data(), sizeof(int64_t) * (n + 1));
        std::memcpy(nU, S.nU.data(), sizeof(int32_t) * n);
        std::memcpy(LUi, S.LUi.data(), sizeof(int32_t) * S.LUi.size());
    }
    return S.nnz();
}

extern "C" int64_t gblu_symmetric_fill(int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *Q)
{
    int64_t fill = 0;
    const int rc = gblu_symmetric_cost(n, Ap, Ai, Q, &fill, nullptr);
    return rc != GBLU_OK ? rc : fill;
}

extern "C" int gblu_order_mindeg(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm)
{
    std::string err;
    if (validate_pattern(n, Ap, Ai, err) != GBLU_OK || !perm) return GBLU_ERR_INVALID_INPUT;
    mindeg_order(n, Ap, Ai, perm);
    return GBLU_OK;
}

extern "C" int32_t gblu_solve_partition(int32_t n, const int64_t *count_from, const int64_t *rowlen,
                                        double density, double frac, long long min_entries, int slices,
                                        int max_piece, int32_t *cut, int32_t *ncut)
{
    if (n < 1 || !count_from || !rowlen || !cut || !ncut || slices < 0 || max_piece < 1 || frac < 0.0 ||
        density < 0.0)
        return record_error(GBLU_ERR_INVALID_INPUT, "solve partition: invalid arguments");
    SolveSplit sp;
    sp.density = density;
    sp.frac = frac;
    sp.min_entries = min_entries;
    sp.slices = slices;
    sp.max_piece = max_piece;
    std::vector<int64_t> cf(count_from, count_from + n + 1), rl(rowlen, rowlen + n);
    std::vector<int32_t> c;
    const int32_t p0 = dense_split(n, cf, rl, sp, c);
    std::copy(c.begin(), c.end(), cut);
    *ncut = (int32_t)c.size();
    return p0;
}

extern "C" int gblu_order_amf(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm)
{
    std::string err;
    if (validate_pattern(n, Ap, Ai, err) != GBLU_OK || !perm)
        return record_error(GBLU_ERR_INVALID_INPUT, "order_amf: invalid pattern or null perm");
    mindeg_order(n, Ap, Ai, perm, nullptr, true);
    return GBLU_OK;
}

extern "C" int gblu_order_cmd(int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *group, int32_t *perm)
{
    std::string err;
    if (validate_pattern(n, Ap, Ai, err) != GBLU_OK || !perm || !group)
        return record_error(GBLU_ERR_INVALID_INPUT, "order_cmd: invalid pattern or null array");
    for (int32_t i = 0; i < n; i++)
        if (group[i] < 0) return record_error(GBLU_ERR_INVALID_INPUT, "order_cmd: negative group");
    mindeg_order(n, Ap, Ai, perm, group);
    return GBLU_OK;
}
