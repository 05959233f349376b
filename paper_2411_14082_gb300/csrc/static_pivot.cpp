// Static pivoting and scaling (the optional pre-processing of Section III-A):
// a row permutation that puts large entries on the diagonal and row and
// column scalings that make those entries 1 and every other entry at most 1
// in magnitude.
//
// The permutation maximizes the product of the diagonal magnitudes.  With
// cmax_j = max_i |a_ij| and c_ij = log(cmax_j / |a_ij|) >= 0 on the nonzero
// entries, that is a minimum-cost perfect matching of columns to rows.  It
// is found by successive shortest augmenting paths with dual potentials:
// u (rows) and v (columns) keep every reduced cost r_ij = c_ij - u_i - v_j
// nonnegative and the matched edges at zero; each augmentation runs
// Dijkstra on the reduced costs from a free column until it settles a free
// row, then shifts the potentials of the settled nodes and flips the path.
// At the end the duals give the scalings: with Dr_i = exp(u_i) and
// Dc_j = exp(v_j) / cmax_j, |Dr_i a_ij Dc_j| = exp(-r_ij) <= 1, and = 1 on
// the matching.  A pattern without a perfect matching on its nonzero
// entries is structurally singular.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <functional>
#include <limits>
#include <queue>
#include <string>
#include <utility>
#include <vector>

#include "gblu_internal.h"

namespace {

constexpr double kInf = std::numeric_limits<double>::infinity();

}  // namespace

extern "C" int gblu_static_pivot(int32_t n, const int32_t *Ap, const int32_t *Ai, const double *Ax,
                                 int32_t *match, double *row_scale, double *col_scale)
{
    std::string err;
    if (gblu::validate_pattern(n, Ap, Ai, err) != GBLU_OK)
        return gblu::record_error(GBLU_ERR_INVALID_INPUT, ("static pivot: invalid pattern: " + err).c_str());
    if (!Ax || !match) return gblu::record_error(GBLU_ERR_INVALID_INPUT, "static pivot: null array");
    // costs on the nonzero entries
    std::vector<double> cost(Ap[n]), lcmax(n, -kInf);
    for (int32_t j = 0; j < n; j++)
        for (int32_t e = Ap[j]; e < Ap[j + 1]; e++)
            if (Ax[e] != 0.0) lcmax[j] = std::max(lcmax[j], std::log(std::fabs(Ax[e])));
    for (int32_t j = 0; j < n; j++) {
        if (!(lcmax[j] > -kInf))
            return gblu::record_error(GBLU_ERR_SINGULAR, "static pivot: a column has no nonzero entry");
        for (int32_t e = Ap[j]; e < Ap[j + 1]; e++)
            cost[e] = Ax[e] != 0.0 ? lcmax[j] - std::log(std::fabs(Ax[e])) : kInf;
    }
    // column reduction, then a greedy matching on the zero reduced costs
    std::vector<double> u(n, 0.0), v(n, 0.0);
    std::vector<int32_t> mrow(n, -1), mcol(n, -1);   // row -> column, column -> row
    for (int32_t j = 0; j < n; j++) {
        double m = kInf;
        for (int32_t e = Ap[j]; e < Ap[j + 1]; e++) m = std::min(m, cost[e]);
        v[j] = m;
        for (int32_t e = Ap[j]; e < Ap[j + 1]; e++) {
            const int32_t i = Ai[e];
            if (cost[e] == m && mrow[i] < 0) {
                mrow[i] = j;
                mcol[j] = i;
                break;
            }
        }
    }
    // shortest augmenting paths from every free column
    std::vector<double> drow(n, kInf), dcol(n, kInf);
    std::vector<int32_t> pred(n, -1);   // row -> column it was reached from
    std::vector<int32_t> touched_r, settled_r, settled_c;
    std::vector<uint8_t> done_r(n, 0);
    using Item = std::pair<double, int32_t>;
    for (int32_t j0 = 0; j0 < n; j0++) {
        if (mcol[j0] >= 0) continue;
        std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
        touched_r.clear();
        settled_r.clear();
        settled_c.clear();
        dcol[j0] = 0.0;
        settled_c.push_back(j0);
        int32_t jc = j0, free_row = -1;
        double L = kInf;
        for (;;) {
            // relax the edges of column jc
            for (int32_t e = Ap[jc]; e < Ap[jc + 1]; e++) {
                const int32_t i = Ai[e];
                if (done_r[i] || !(cost[e] < kInf)) continue;
                const double d = dcol[jc] + (cost[e] - u[i] - v[jc]);
                if (d < drow[i]) {
                    if (drow[i] == kInf) touched_r.push_back(i);
                    drow[i] = d;
                    pred[i] = jc;
                    pq.push({d, i});
                }
            }
            // settle the nearest row
            int32_t i = -1;
            while (!pq.empty()) {
                const Item it = pq.top();
                pq.pop();
                if (done_r[it.second] || it.first > drow[it.second]) continue;
                i = it.second;
                break;
            }
            if (i < 0) break;   // no free row reachable
            done_r[i] = 1;
            if (mrow[i] < 0) {
                free_row = i;
                L = drow[i];
                break;
            }
            settled_r.push_back(i);
            jc = mrow[i];
            dcol[jc] = drow[i];   // the matched edge has reduced cost 0
            settled_c.push_back(jc);
        }
        if (free_row < 0) {
            return gblu::record_error(GBLU_ERR_SINGULAR, "static pivot: the pattern has no perfect matching "
                                                         "on its nonzero entries (structurally singular)");
        }
        // potentials: settled nodes move by L - distance, which keeps every
        // reduced cost >= 0 and makes the path edges tight
        for (int32_t j : settled_c) v[j] += L - dcol[j];
        for (int32_t r : settled_r) u[r] -= L - drow[r];
        // flip the path
        int32_t i = free_row;
        while (i >= 0) {
            const int32_t j = pred[i];
            const int32_t next = mcol[j];
            mrow[i] = j;
            mcol[j] = i;
            i = (j == j0) ? -1 : next;
        }
        for (int32_t r : touched_r) {
            drow[r] = kInf;
            done_r[r] = 0;
            pred[r] = -1;
        }
        for (int32_t j : settled_c) dcol[j] = kInf;
    }
    for (int32_t j = 0; j < n; j++) match[j] = mcol[j];
    if (row_scale)
        for (int32_t i = 0; i < n; i++) row_scale[i] = std::exp(u[i]);
    if (col_scale)
        for (int32_t j = 0; j < n; j++) col_scale[j] = std::exp(v[j] - lcmax[j]);
    return GBLU_OK;
}

extern "C" int gblu_permute_rows(int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *match,
                                 int32_t *Ai_out, int32_t *src_out)
{
    std::string err;
    if (gblu::validate_pattern(n, Ap, Ai, err) != GBLU_OK || !match || !Ai_out || !src_out)
        return gblu::record_error(GBLU_ERR_INVALID_INPUT, "permute rows: invalid pattern or null array");
    std::vector<int32_t> newrow(n, -1);
    for (int32_t j = 0; j < n; j++) {
        if (match[j] < 0 || match[j] >= n || newrow[match[j]] >= 0)
            return gblu::record_error(GBLU_ERR_INVALID_INPUT, "permute rows: match is not a permutation");
        newrow[match[j]] = j;
    }
    std::vector<std::pair<int32_t, int32_t>> col;
    for (int32_t j = 0; j < n; j++) {
        col.clear();
        for (int32_t e = Ap[j]; e < Ap[j + 1]; e++) col.push_back({newrow[Ai[e]], e});
        std::sort(col.begin(), col.end());
        for (size_t t = 0; t < col.size(); t++) {
            Ai_out[Ap[j] + t] = col[t].first;
            src_out[Ap[j] + t] = col[t].second;
        }
    }
    return GBLU_OK;
}
