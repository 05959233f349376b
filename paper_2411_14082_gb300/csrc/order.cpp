// Minimum-degree fill-reducing ordering on the pattern of A + A^T
// (pre-processing, Section III-A; the paper uses approximate minimum degree).
//
// Quotient-graph elimination: eliminating variable p turns it into an
// element whose variable set Lp is the union of p's variable neighbours and
// of the variable sets of p's element neighbours; those elements are
// absorbed.  The degree of every variable i in Lp is then bounded by
//     |A_i| + (|Lp| - 1) + sum over other elements e of i of |L_e \ Lp|,
// the approximate external degree of Amestoy, Davis and Duff (1996).
// Elements contained in Lp are absorbed as well.  Ties go to the lower
// index, so the order is deterministic.
//
// Constrained form (the constrained minimum degree that Section III-A
// applies after an incomplete nested dissection): every variable carries a
// group number and the pivot is the variable of least degree among those of
// the lowest group still present, so groups are eliminated in order while
// the degrees still see the whole graph.
//
// Deficiency form (the approximate minimum deficiency variant Section III-A
// also runs): the pivot is the variable whose elimination is estimated to
// create the fewest new entries, d(d-1)/2 - c(c-1)/2, where d is its
// approximate degree and c+1 the size of the largest element it belongs to
// (the pairs of that clique exist already); the approximate mean local fill
// score of Rothberg and Eisenstat.
#include <algorithm>
#include <functional>
#include <queue>
#include <vector>

#include "gblu_internal.h"

namespace gblu {

void mindeg_order(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm, const int32_t *group,
                  bool deficiency)
{
    std::vector<std::vector<int32_t>> A(n), E(n), Lel(n);
    for (int32_t c = 0; c < n; c++)
        for (int32_t p = Ap[c]; p < Ap[c + 1]; p++) {
            const int32_t r = Ai[p];
            if (r == c) continue;
            A[r].push_back(c);
            A[c].push_back(r);
        }
    for (int32_t i = 0; i < n; i++) {
        std::sort(A[i].begin(), A[i].end());
        A[i].erase(std::unique(A[i].begin(), A[i].end()), A[i].end());
    }
    std::vector<char> elim(n, 0), alive(n, 0);
    std::vector<int32_t> mark(n, -1), wmark(n, -1);
    std::vector<int64_t> w(n, 0), score(n);
    // key: group, then the score (degree, or estimated fill); ties by index
    constexpr int64_t kScoreMax = INT64_MAX / 4;
    using Key = std::pair<int32_t, int64_t>;
    auto key = [&](int32_t i) { return Key{group ? group[i] : 0, score[i]}; };
    auto score_of = [&](int64_t d, int64_t c) -> int64_t {
        if (!deficiency) return d;
        c = std::min(c, d);
        return std::min(kScoreMax, (d * (d - 1) - c * (c - 1)) / 2);
    };
    // min-heap of (key, variable) with lazy deletion: an update pushes a new
    // entry, and a popped entry counts only if it still holds the variable's
    // key; the first valid entry is the least (key, index) pair, as in an
    // ordered set.  Rebuilt from the live variables when stale entries pile up.
    using Entry = std::pair<Key, int32_t>;
    std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> pq;
    for (int32_t i = 0; i < n; i++) {
        score[i] = score_of((int64_t)A[i].size(), 0);
        pq.push({key(i), i});
    }
    std::vector<int32_t> Lp;
    for (int32_t k = 0; k < n; k++) {
        while (elim[pq.top().second] || pq.top().first != key(pq.top().second)) pq.pop();
        const int32_t p = pq.top().second;
        pq.pop();
        perm[k] = p;
        elim[p] = 1;
        // ---- element p: Lp = variables adjacent to p directly or via elements
        Lp.clear();
        mark[p] = k;
        for (int32_t v : A[p])
            if (!elim[v] && mark[v] != k) { mark[v] = k; Lp.push_back(v); }
        for (int32_t e : E[p]) {
            if (!alive[e]) continue;
            for (int32_t v : Lel[e])
                if (!elim[v] && mark[v] != k) { mark[v] = k; Lp.push_back(v); }
            alive[e] = 0;  // absorbed into p
            std::vector<int32_t>().swap(Lel[e]);
        }
        std::vector<int32_t>().swap(A[p]);
        std::vector<int32_t>().swap(E[p]);
        Lel[p] = Lp;
        alive[p] = 1;
        // ---- |L_e \ Lp| for the other elements next to Lp
        for (int32_t i : Lp)
            for (int32_t e : E[i]) {
                if (!alive[e] || e == p) continue;
                if (wmark[e] != k) { wmark[e] = k; w[e] = (int64_t)Lel[e].size(); }
                w[e]--;
            }
        // ---- update the variables of Lp
        const int32_t remaining = n - k - 1;
        for (int32_t i : Lp) {
            std::vector<int32_t> &Ei = E[i];
            size_t o = 0;
            int64_t ext = 0, clique = (int64_t)Lp.size() - 1;
            for (int32_t e : Ei) {
                if (!alive[e] || e == p) continue;
                if (wmark[e] == k && w[e] <= 0) {  // e inside Lp: absorb
                    alive[e] = 0;
                    std::vector<int32_t>().swap(Lel[e]);
                    continue;
                }
                Ei[o++] = e;
                ext += (wmark[e] == k) ? w[e] : (int64_t)Lel[e].size();
                clique = std::max(clique, (int64_t)Lel[e].size() - 1);
            }
            Ei.resize(o);
            Ei.push_back(p);
            std::vector<int32_t> &Ai_ = A[i];
            size_t q = 0;
            for (int32_t v : Ai_)
                if (!elim[v] && mark[v] != k && v != i) Ai_[q++] = v;
            Ai_.resize(q);
            int64_t d = (int64_t)Ai_.size() + (int64_t)Lp.size() - 1 + ext;
            if (d > remaining - 1) d = remaining - 1;
            if (d < 0) d = 0;
            const int64_t s = score_of(d, clique);
            if (s != score[i]) {
                score[i] = s;
                pq.push({key(i), i});
            }
        }
        if (pq.size() > (size_t)4 * (size_t)(n - k) + 1024) {
            std::vector<Entry> live;
            live.reserve(n - k);
            for (int32_t v = 0; v < n; v++)
                if (!elim[v]) live.push_back({key(v), v});
            pq = std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>>(std::greater<Entry>(),
                                                                                     std::move(live));
        }
    }
}

}  // namespace gblu
