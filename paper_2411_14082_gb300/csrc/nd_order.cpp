// Nested dissection ordering of a general sparse pattern (the fill-reducing
// ordering family of Section III-A for mesh-like matrices), without
// coordinates.
//
// The graph is that of A + A^T without the diagonal.  A vertex set is split
// by a vertex separator, the two halves are ordered recursively and the
// separator is numbered after both; small sets (and sets that do not split
// well) are ordered by minimum degree.  Each split is multilevel:
//   coarsen  - heavy-edge matching, repeated until the graph is small;
//   bisect   - greedy graph growing from a few seeds on the coarsest graph,
//              keeping the smallest edge cut with balanced vertex weight;
//   refine   - projected back level by level, each level improved by
//              Fiduccia-Mattheyses passes (moves of the largest gain, also
//              negative, under the balance bound; rollback to the best cut);
//   separate - a vertex cover of the cut edges (greedy, endpoint with more
//              cut edges first) becomes the separator; separator vertices
//              with no neighbour on one side then leave it.
// Each split keeps the smallest of three trials (twelve at the two top
// levels, whose separators become the largest dense blocks).  Every node of
// the dissection tree draws from its own generator, seeded from its
// parent's, and the subtrees of the top four levels run on threads of their
// own: the ordering is deterministic and independent of thread timing.
//
// Constrained form (Section III-A's incomplete nested dissection followed by
// constrained minimum degree): the same dissection only numbers groups, each
// leaf set and then each separator after its two halves, and one
// constrained minimum-degree pass orders the whole graph group by group, so
// the leaves' orders see their boundaries and the separators are ordered
// too.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <queue>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "gblu_internal.h"

namespace {

struct Graph {
    int32_t n = 0;
    std::vector<int64_t> ptr;
    std::vector<int32_t> adj, ew;   // neighbours and edge weights
    std::vector<int32_t> vw;        // vertex weights
    int64_t total_w() const { return std::accumulate(vw.begin(), vw.end(), int64_t(0)); }
};

// the graph induced by `verts` (global ids) in the global graph g
Graph induced(const Graph &g, const std::vector<int32_t> &verts, std::vector<int32_t> &local)
{
    Graph s;
    s.n = (int32_t)verts.size();
    for (int32_t i = 0; i < s.n; i++) local[verts[i]] = i;
    s.ptr.assign(s.n + 1, 0);
    for (int32_t i = 0; i < s.n; i++) {
        const int32_t v = verts[i];
        for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; e++)
            if (local[g.adj[e]] >= 0) {
                s.adj.push_back(local[g.adj[e]]);
                s.ew.push_back(1);
            }
        s.ptr[i + 1] = (int64_t)s.adj.size();
    }
    s.vw.assign(s.n, 1);
    for (int32_t v : verts) local[v] = -1;
    return s;
}

// heavy-edge matching; cmap[v] = coarse vertex of v
Graph coarsen(const Graph &g, std::vector<int32_t> &cmap, std::mt19937 &rng)
{
    std::vector<int32_t> order(g.n), match(g.n, -1);
    std::iota(order.begin(), order.end(), 0);
    std::shuffle(order.begin(), order.end(), rng);
    for (int32_t v : order) {
        if (match[v] >= 0) continue;
        int32_t best = -1, bw = -1;
        for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; e++) {
            const int32_t u = g.adj[e];
            if (u != v && match[u] < 0 && g.ew[e] > bw) {
                bw = g.ew[e];
                best = u;
            }
        }
        if (best >= 0) {
            match[v] = best;
            match[best] = v;
        } else {
            match[v] = v;
        }
    }
    cmap.assign(g.n, -1);
    int32_t nc = 0;
    for (int32_t v = 0; v < g.n; v++) {
        if (cmap[v] >= 0) continue;
        cmap[v] = nc;
        cmap[match[v]] = nc;
        nc++;
    }
    Graph c;
    c.n = nc;
    c.vw.assign(nc, 0);
    for (int32_t v = 0; v < g.n; v++) c.vw[cmap[v]] += g.vw[v];
    std::vector<std::vector<int32_t>> members(nc);
    for (int32_t v = 0; v < g.n; v++) members[cmap[v]].push_back(v);
    std::vector<int32_t> slot(nc, -1);
    c.ptr.assign(nc + 1, 0);
    for (int32_t cv = 0; cv < nc; cv++) {
        const int64_t start = (int64_t)c.adj.size();
        for (int32_t v : members[cv])
            for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; e++) {
                const int32_t cu = cmap[g.adj[e]];
                if (cu == cv) continue;
                if (slot[cu] < 0) {
                    slot[cu] = (int32_t)c.adj.size();
                    c.adj.push_back(cu);
                    c.ew.push_back(g.ew[e]);
                } else {
                    c.ew[slot[cu]] += g.ew[e];
                }
            }
        for (int64_t e = start; e < (int64_t)c.adj.size(); e++) slot[c.adj[e]] = -1;
        c.ptr[cv + 1] = (int64_t)c.adj.size();
    }
    return c;
}

int64_t cut_of(const Graph &g, const std::vector<uint8_t> &part)
{
    int64_t cut = 0;
    for (int32_t v = 0; v < g.n; v++)
        for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; e++)
            if (part[v] != part[g.adj[e]]) cut += g.ew[e];
    return cut / 2;
}

// greedy graph growing from `seeds` random starts: part 0 grows by BFS
// until it holds half of the vertex weight
std::vector<uint8_t> grow_bisect(const Graph &g, std::mt19937 &rng, int seeds)
{
    const int64_t W = g.total_w();
    std::vector<uint8_t> best(g.n, 0);
    int64_t best_cut = -1;
    std::vector<uint8_t> part(g.n);
    std::vector<int32_t> queue;
    std::uniform_int_distribution<int32_t> pick(0, g.n - 1);
    for (int s = 0; s < seeds; s++) {
        std::fill(part.begin(), part.end(), 1);
        int64_t w0 = 0;
        queue.clear();
        std::vector<uint8_t> seen(g.n, 0);
        int32_t head = 0;
        int32_t start = pick(rng);
        queue.push_back(start);
        seen[start] = 1;
        while (w0 * 2 < W) {
            if (head == (int32_t)queue.size()) {   // another component: restart from an unseen vertex
                int32_t u = -1;
                for (int32_t t = 0; t < g.n; t++)
                    if (!seen[t]) {
                        u = t;
                        break;
                    }
                if (u < 0) break;
                seen[u] = 1;
                queue.push_back(u);
            }
            const int32_t v = queue[head++];
            part[v] = 0;
            w0 += g.vw[v];
            for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; e++) {
                const int32_t u = g.adj[e];
                if (!seen[u]) {
                    seen[u] = 1;
                    queue.push_back(u);
                }
            }
        }
        const int64_t c = cut_of(g, part);
        if (best_cut < 0 || c < best_cut) {
            best_cut = c;
            best = part;
        }
    }
    return best;
}

// Fiduccia-Mattheyses passes: repeatedly move the unlocked vertex of
// largest cut gain (negative gains too) whose move keeps both sides within
// [lo, hi] of the vertex weight, lock it, and at the end of the pass roll
// back to the smallest cut seen
void refine(const Graph &g, std::vector<uint8_t> &part, int passes)
{
    const int64_t W = g.total_w();
    const int64_t lo = (int64_t)(0.40 * (double)W), hi = W - lo;
    std::vector<int64_t> gain(g.n);
    std::vector<uint8_t> locked(g.n);
    using Item = std::pair<int64_t, int32_t>;
    for (int p = 0; p < passes; p++) {
        int64_t w0 = 0, cut = 0;
        for (int32_t v = 0; v < g.n; v++) {
            if (part[v] == 0) w0 += g.vw[v];
            int64_t ext = 0, in = 0;
            for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; e++)
                (part[g.adj[e]] != part[v] ? ext : in) += g.ew[e];
            gain[v] = ext - in;
            cut += ext;
        }
        cut /= 2;
        std::priority_queue<Item> pq;
        for (int32_t v = 0; v < g.n; v++) {
            locked[v] = 0;
            bool boundary = false;
            for (int64_t e = g.ptr[v]; e < g.ptr[v + 1] && !boundary; e++) boundary = part[g.adj[e]] != part[v];
            if (boundary) pq.push({gain[v], v});
        }
        std::vector<int32_t> moves;
        int64_t best_cut = cut, cur = cut;
        size_t best_len = 0;
        const size_t limit = std::max<size_t>(64, (size_t)g.n / 50);
        while (!pq.empty()) {
            const Item it = pq.top();
            pq.pop();
            const int32_t v = it.second;
            if (locked[v] || it.first != gain[v]) continue;
            const int64_t nw0 = part[v] == 0 ? w0 - g.vw[v] : w0 + g.vw[v];
            if (nw0 < lo || nw0 > hi) continue;
            locked[v] = 1;
            part[v] ^= 1;
            w0 = nw0;
            cur -= gain[v];
            moves.push_back(v);
            for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; e++) {
                const int32_t u = g.adj[e];
                if (locked[u]) continue;
                gain[u] += (part[u] == part[v]) ? -2 * (int64_t)g.ew[e] : 2 * (int64_t)g.ew[e];
                pq.push({gain[u], u});
            }
            if (cur < best_cut) {
                best_cut = cur;
                best_len = moves.size();
            } else if (moves.size() - best_len > limit) {
                break;
            }
        }
        for (size_t k = moves.size(); k-- > best_len;) part[moves[k]] ^= 1;
        if (best_len == 0) break;
    }
}

// multilevel bisection of g
std::vector<uint8_t> bisect(const Graph &g, std::mt19937 &rng)
{
    std::vector<Graph> levels;
    std::vector<std::vector<int32_t>> maps;
    levels.push_back(g);
    while (levels.back().n > 160 && levels.size() < 40) {
        std::vector<int32_t> cmap;
        Graph c = coarsen(levels.back(), cmap, rng);
        if (c.n > (int32_t)(0.95 * levels.back().n)) break;   // matching stalled
        maps.push_back(std::move(cmap));
        levels.push_back(std::move(c));
    }
    std::vector<uint8_t> part = grow_bisect(levels.back(), rng, 8);
    refine(levels.back(), part, 8);
    for (int l = (int)levels.size() - 2; l >= 0; l--) {
        std::vector<uint8_t> fine(levels[l].n);
        for (int32_t v = 0; v < levels[l].n; v++) fine[v] = part[maps[l][v]];
        part.swap(fine);
        refine(levels[l], part, 4);
    }
    return part;
}

// one block of the result, in elimination order: a leaf set (ordered by
// minimum degree in the plain form) or a separator (vertex order)
struct Block {
    std::vector<int32_t> verts;
};

// seed of a child of the dissection-tree node with seed `s` (splitmix64
// finalizer), so that every node draws from its own generator and the
// result does not depend on which thread runs which subtree
uint64_t child_seed(uint64_t s, uint64_t child)
{
    uint64_t z = s + 0x9E3779B97F4A7C15ULL * (child + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// bisection trials at the dissection tree's top levels
constexpr int kTopDepth = 2, kTopTrials = 12;

struct Ordering {
    const Graph &g;
    int32_t leaf;
    bool constrained;    // leaves keep their vertex order (groups only)
    int par_depth;       // subtrees above this depth run on threads of their own

    void leaf_block(std::vector<int32_t> &&verts, std::vector<int32_t> &local, std::vector<Block> &out) const
    {
        Block blk;
        if (constrained || verts.size() <= 2) {
            blk.verts = std::move(verts);
        } else {
            Graph s = induced(g, verts, local);
            std::vector<int32_t> Ap(s.ptr.begin(), s.ptr.end()), perm(s.n);
            gblu::mindeg_order(s.n, Ap.data(), s.adj.data(), perm.data());
            blk.verts.resize(s.n);
            for (int32_t i = 0; i < s.n; i++) blk.verts[i] = verts[perm[i]];
        }
        out.push_back(std::move(blk));
    }

    // vertex separator of a bisection: side[v] = 0 / 1, or 2 for the separator
    static std::vector<uint8_t> separate(const Graph &s, const std::vector<uint8_t> &part)
    {
        // a vertex cover of the cut edges, endpoint with more cut edges first
        std::vector<int32_t> cdeg(s.n, 0);
        for (int32_t v = 0; v < s.n; v++)
            for (int64_t e = s.ptr[v]; e < s.ptr[v + 1]; e++)
                if (part[v] != part[s.adj[e]]) cdeg[v]++;
        std::vector<int32_t> byc;
        for (int32_t v = 0; v < s.n; v++)
            if (cdeg[v] > 0) byc.push_back(v);
        std::sort(byc.begin(), byc.end(), [&](int32_t a, int32_t b) { return cdeg[a] != cdeg[b] ? cdeg[a] > cdeg[b] : a < b; });
        std::vector<uint8_t> side(part.begin(), part.end());
        for (int32_t v : byc) {
            bool needed = false;   // an uncovered cut edge left at v
            for (int64_t e = s.ptr[v]; e < s.ptr[v + 1]; e++) {
                const int32_t u = s.adj[e];
                if (side[u] != 2 && side[u] != side[v] && side[v] != 2) {
                    needed = true;
                    break;
                }
            }
            if (needed) side[v] = 2;
        }
        // refinement: a separator vertex with no neighbour on one side
        // joins the other side (repeat while that shrinks the separator)
        for (int pass = 0; pass < 8; pass++) {
            int moved = 0;
            int64_t w[2] = {0, 0};
            for (int32_t v = 0; v < s.n; v++)
                if (side[v] < 2) w[side[v]] += s.vw[v];
            for (int32_t v = 0; v < s.n; v++) {
                if (side[v] != 2) continue;
                bool has[2] = {false, false};
                for (int64_t e = s.ptr[v]; e < s.ptr[v + 1]; e++)
                    if (side[s.adj[e]] < 2) has[side[s.adj[e]]] = true;
                if (has[0] && has[1]) continue;
                const int to = !has[0] && !has[1] ? (w[0] <= w[1] ? 0 : 1) : (has[0] ? 0 : 1);
                side[v] = (uint8_t)to;
                w[to] += s.vw[v];
                moved++;
            }
            if (!moved) break;
        }
        return side;
    }

    // blocks of `verts` in elimination order: the two halves' blocks, then
    // the separator.  local: scratch of n entries, all -1, owned by the
    // calling thread.
    void rec(std::vector<int32_t> verts, int depth, uint64_t seed, std::vector<int32_t> &local,
             std::vector<Block> &out) const
    {
        if ((int32_t)verts.size() <= leaf || depth > 60) {
            leaf_block(std::move(verts), local, out);
            return;
        }
        Graph s = induced(g, verts, local);
        std::mt19937 rng{(uint32_t)(seed ^ (seed >> 32))};
        // a few multilevel trials (more near the root, whose separators
        // become the largest dense blocks); keep the smallest separator
        std::vector<uint8_t> side;
        int64_t best = -1;
        const int trials = depth < kTopDepth ? kTopTrials : 3;
        for (int t = 0; t < trials; t++) {
            std::vector<uint8_t> sd = separate(s, bisect(s, rng));
            int64_t ns = 0, n0 = 0, n1 = 0;
            for (uint8_t x : sd) (x == 2 ? ns : x == 0 ? n0 : n1)++;
            if (n0 == 0 || n1 == 0) continue;
            if (best < 0 || ns < best) {
                best = ns;
                side.swap(sd);
            }
        }
        if (best < 0) {
            leaf_block(std::move(verts), local, out);
            return;
        }
        std::vector<int32_t> a, b, sep;
        for (int32_t v = 0; v < s.n; v++) (side[v] == 2 ? sep : side[v] == 0 ? a : b).push_back(verts[v]);
        if (a.empty() || b.empty() || sep.size() * 3 > verts.size()) {   // no useful split
            leaf_block(std::move(verts), local, out);
            return;
        }
        std::vector<int32_t>().swap(verts);
        if (depth < par_depth) {
            // the first half on a thread of its own, with its own scratch
            std::vector<Block> out_a;
            std::thread ta([&]() {
                std::vector<int32_t> local_a(g.n, -1);
                rec(std::move(a), depth + 1, child_seed(seed, 0), local_a, out_a);
            });
            std::vector<Block> out_b;
            rec(std::move(b), depth + 1, child_seed(seed, 1), local, out_b);
            ta.join();
            for (Block &x : out_a) out.push_back(std::move(x));
            for (Block &x : out_b) out.push_back(std::move(x));
        } else {
            rec(std::move(a), depth + 1, child_seed(seed, 0), local, out);
            rec(std::move(b), depth + 1, child_seed(seed, 1), local, out);
        }
        out.push_back(Block{std::move(sep)});
    }
};

}  // namespace

namespace gblu {

void nd_order(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm, int32_t leaf, bool constrained)
{
    Graph g;
    g.n = n;
    std::vector<std::vector<int32_t>> nb(n);
    for (int32_t c = 0; c < n; c++)
        for (int32_t p = Ap[c]; p < Ap[c + 1]; p++) {
            const int32_t r = Ai[p];
            if (r == c) continue;
            nb[r].push_back(c);
            nb[c].push_back(r);
        }
    g.ptr.assign(n + 1, 0);
    for (int32_t v = 0; v < n; v++) {
        std::sort(nb[v].begin(), nb[v].end());
        nb[v].erase(std::unique(nb[v].begin(), nb[v].end()), nb[v].end());
        g.adj.insert(g.adj.end(), nb[v].begin(), nb[v].end());
        g.ptr[v + 1] = (int64_t)g.adj.size();
        std::vector<int32_t>().swap(nb[v]);
    }
    g.ew.assign(g.adj.size(), 1);
    g.vw.assign(n, 1);
    // up to 2^kParDepth subtrees on threads of their own
    constexpr int kParDepth = 4;
    const Ordering o{g, leaf, constrained, kParDepth};
    std::vector<int32_t> all(n), local(n, -1);
    std::iota(all.begin(), all.end(), 0);
    std::vector<Block> blocks;
    o.rec(std::move(all), 0, 20241121u, local, blocks);
    if (constrained) {
        // groups in block order: each leaf set, then each separator after
        // its two halves
        std::vector<int32_t> grp(n, 0);
        for (size_t b = 0; b < blocks.size(); b++)
            for (int32_t v : blocks[b].verts) grp[v] = (int32_t)b;
        mindeg_order(n, Ap, Ai, perm, grp.data());
        return;
    }
    int32_t k = 0;
    for (const Block &b : blocks)
        for (int32_t v : b.verts) perm[k++] = v;
}

// Section III-A runs several orderings and keeps the best.  Candidates here:
// minimum degree and approximate minimum deficiency (up to kAutoMindegMax
// unknowns; on the 200x200x4 mesh they take 4.5 and 2.2 s and cost 5x and
// 2x the flops of dissection, but circuits without mesh structure can
// favour them), nested
// dissection, and incomplete nested dissection with constrained minimum
// degree (up to kAutoCndMax unknowns: its minimum-degree pass over the
// whole graph costs about 2.2x the dissection at 360,000 unknowns for a
// 0.25% gain), each on a host thread of its own.  The one
// whose factorization costs the fewest flops when every diagonal pivot is
// kept (F = sum_j 2 c_j^2 of the symmetric pattern, the re-factorization's
// work) wins; ties go to the earlier candidate.
int auto_order(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm)
{
    constexpr int32_t kAutoMindegMax = 200000, kAutoCndMax = 200000;
    struct Candidate {
        int method;
        std::vector<int32_t> perm;
        double flops = 0.0;
    };
    std::vector<Candidate> cand;
    if (n <= kAutoMindegMax) {
        cand.push_back({GBLU_ORDER_MINDEG, {}, 0.0});
        cand.push_back({GBLU_ORDER_AMF, {}, 0.0});
    }
    cand.push_back({GBLU_ORDER_ND, {}, 0.0});
    if (n <= kAutoCndMax) cand.push_back({GBLU_ORDER_CND, {}, 0.0});
    auto run = [n, Ap, Ai](Candidate *c) {
        c->perm.resize(n);
        if (c->method == GBLU_ORDER_MINDEG || c->method == GBLU_ORDER_AMF)
            mindeg_order(n, Ap, Ai, c->perm.data(), nullptr, c->method == GBLU_ORDER_AMF);
        else
            nd_order(n, Ap, Ai, c->perm.data(), 256, c->method == GBLU_ORDER_CND);
        Pattern P;
        P.n = n;
        P.Ap.assign(Ap, Ap + n + 1);
        P.Ai.assign(Ai, Ai + Ap[n]);
        P.Q = c->perm;
        P.qinv.assign(n, 0);
        for (int32_t k = 0; k < n; k++) P.qinv[c->perm[k]] = k;
        symmetric_fill(P, &c->flops);
    };
    std::vector<std::thread> th;
    for (size_t i = 1; i < cand.size(); i++) th.emplace_back(run, &cand[i]);
    run(&cand[0]);
    for (std::thread &t : th) t.join();
    size_t best = 0;
    for (size_t i = 1; i < cand.size(); i++)
        if (cand[i].flops < cand[best].flops) best = i;
    std::copy(cand[best].perm.begin(), cand[best].perm.end(), perm);
    return cand[best].method;
}

}  // namespace gblu

extern "C" int gblu_order_auto(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm, int32_t *method)
{
    std::string err;
    if (gblu::validate_pattern(n, Ap, Ai, err) != GBLU_OK || !perm)
        return gblu::record_error(GBLU_ERR_INVALID_INPUT, "order_auto: invalid pattern or null perm");
    const int m = gblu::auto_order(n, Ap, Ai, perm);
    if (method) *method = m;
    return GBLU_OK;
}

extern "C" int gblu_order_nd(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm)
{
    std::string err;
    if (gblu::validate_pattern(n, Ap, Ai, err) != GBLU_OK || !perm)
        return gblu::record_error(GBLU_ERR_INVALID_INPUT, "order_nd: invalid pattern or null perm");
    gblu::nd_order(n, Ap, Ai, perm, 256);
    return GBLU_OK;
}

extern "C" int gblu_order_cnd(int32_t n, const int32_t *Ap, const int32_t *Ai, int32_t *perm)
{
    std::string err;
    if (gblu::validate_pattern(n, Ap, Ai, err) != GBLU_OK || !perm)
        return gblu::record_error(GBLU_ERR_INVALID_INPUT, "order_cnd: invalid pattern or null perm");
    gblu::nd_order(n, Ap, Ai, perm, 256, true);
    return GBLU_OK;
}
