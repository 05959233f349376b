"""Element-wise comparison of exported GPU factors with oracle factors.

Tolerance.  Column k of L and U comes from one work vector x_k (U(:,k) =
x_k on the pivotal rows, L(:,k) = x_k / U(k,k) on the others).  With
M = |L_o| |U_o| (the magnitudes summed into each entry) and
X_k = max(max|U_o(:,k)|, |U_o(k,k)| * max|L_o(:,k)|) (the largest entry of
x_k), the bound is
    |U_g(i,k) - U_o(i,k)| <= rtol * max(M(i,k), X_k)
    |L_g(i,k) - L_o(i,k)| <= rtol * max(M(i,k), X_k) / |U_o(k,k)|
i.e. every computed work-vector entry agrees to rtol relative to the larger
of its componentwise magnitude and the largest entry of its column.  Entries
that are rounding noise around an exact zero (cancellation) differ between
two valid summation orders by far more than their own size; the column
scale keeps them comparable.

The strict per-column metric is reported beside it:
    ||L_g(:,k) - L_o(:,k)||_inf / ||L_o(:,k)||_inf   (the same for U)
and asserted (<= rtol) on every column above the cancellation noise floor,
i.e. whose inf-norm (for L, times |U(k,k)|) is at least 1e-3 of the largest
|L||U| magnitude summed into it: such a column lost at most three digits to
cancellation, so rounding differences cannot reach rtol in it.
"""
import numpy as np
import scipy.sparse as sp


def _keys(p, i, n):
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(np.asarray(p, dtype=np.int64)))
    return cols * n + np.asarray(i, dtype=np.int64), cols


def abs_product(lu):
    """|L| |U| of the oracle factors as (keys, values) sorted by key."""
    n = lu.n
    L = sp.csc_matrix((np.abs(lu.Lx), lu.Li, lu.Lp), shape=(n, n)) + sp.identity(n, format="csc")
    U = sp.csc_matrix((np.abs(lu.Ux), lu.Ui, lu.Up), shape=(n, n))
    if n <= 2500:
        M = sp.csc_matrix(L.toarray() @ U.toarray())
    else:
        M = (L @ U).tocsc()
    M.sort_indices()
    k, _ = _keys(M.indptr, M.indices, n)
    return k, M.data


NOISE_FLOOR = 1e-3
LOG = []   # one dict per compare_factors call (printed by tests run with -s)


def compare_part(n, gp, gi, gx, op, oi, ox, scale_of, mag_of=None, colmul=None):
    """Oracle entries must all be in the GPU pattern; GPU-only entries must be
    exact zeros.  Returns (max |diff| / scale over the oracle entries,
    per-column max |diff|, per-column max |oracle entry|, per-column max
    magnitude from mag_of)."""
    gk, _ = _keys(gp, gi, n)
    ok, ocols = _keys(op, oi, n)
    pos = np.searchsorted(gk, ok)
    assert np.all(pos < len(gk)) and np.array_equal(gk[np.minimum(pos, len(gk) - 1)], ok), \
        "an oracle entry is missing from the GPU pattern"
    extra = np.ones(len(gk), dtype=bool)
    extra[pos] = False
    assert np.all(gx[extra] == 0.0), "GPU-only pattern entries must be exact zeros"
    scale = scale_of(ok, ocols)
    diff = np.abs(gx[pos] - ox)
    err = diff / np.where(scale > 0, scale, 1.0)
    cdiff, cnorm, cmag = np.zeros(n), np.zeros(n), np.zeros(n)
    if len(ok):
        np.maximum.at(cdiff, ocols, diff)
        np.maximum.at(cnorm, ocols, np.abs(ox))
        if mag_of is not None:
            np.maximum.at(cmag, ocols, mag_of(ok))
    return (float(err.max()) if len(err) else 0.0), cdiff, cnorm, cmag


def strict_columns(cdiff, cnorm, cmag, colmul, rtol):
    """Strict per-column errors; columns above the noise floor are asserted."""
    has = cnorm > 0
    rel = np.where(has, cdiff / np.where(has, cnorm, 1.0), 0.0)
    above = has & (cnorm * colmul >= NOISE_FLOOR * cmag)
    worst = float(rel[above].max()) if above.any() else 0.0
    bad = np.nonzero(above & (rel > rtol))[0]
    assert len(bad) == 0, f"strict per-column error {rel[bad].max():.3e} > {rtol} at columns {bad[:10]}"
    return worst, int(above.sum()), int(has.sum()), float(rel.max()) if has.any() else 0.0


def compare_factors(f, lu, rtol=1e-10):
    """Same column order, same pivot sequence, L and U within rtol (componentwise)."""
    n = lu.n
    assert np.array_equal(f["q"], lu.Q)
    assert np.array_equal(f["piv"], lu.piv), \
        f"pivot sequences differ at steps {np.nonzero(f['piv'] != lu.piv)[0][:10]}"
    mk, mv = abs_product(lu)
    udiag = np.abs(lu.Ux[np.asarray(lu.Up[1:], dtype=np.int64) - 1])
    xcol = np.zeros(n)
    if len(lu.Ux):
        np.maximum.at(xcol, np.repeat(np.arange(n), np.diff(lu.Up)), np.abs(lu.Ux))
    if len(lu.Lx):
        np.maximum.at(xcol, np.repeat(np.arange(n), np.diff(lu.Lp)),
                      np.abs(lu.Lx) * udiag[np.repeat(np.arange(n), np.diff(lu.Lp))])

    def m_at(keys):
        # entries whose |L||U| sum is exactly zero are absent from M
        p = np.minimum(np.searchsorted(mk, keys), len(mk) - 1)
        return np.where(mk[p] == keys, mv[p], 0.0) if len(mk) else np.zeros(len(keys))

    el, ldiff, lnorm, lmag = compare_part(n, f["Lp"], f["Li"], f["Lx"], lu.Lp, lu.Li, lu.Lx,
                                          lambda keys, cols: np.maximum(m_at(keys), xcol[cols]) / udiag[cols],
                                          m_at)
    eu, udiff, unorm, umag = compare_part(n, f["Up"], f["Ui"], f["Ux"], lu.Up, lu.Ui, lu.Ux,
                                          lambda keys, cols: np.maximum(m_at(keys), xcol[cols]), m_at)
    assert el <= rtol and eu <= rtol, f"factor mismatch: L {el:.3e}, U {eu:.3e} (tol {rtol})"
    sl = strict_columns(ldiff, lnorm, lmag, udiag, rtol)
    su = strict_columns(udiff, unorm, umag, np.ones(n), rtol)
    rec = dict(n=n, componentwise=max(el, eu), strict_above_floor=max(sl[0], su[0]),
               strict_all=max(sl[3], su[3]), l_cols_checked=sl[1], l_cols=sl[2],
               u_cols_checked=su[1], u_cols=su[2])
    LOG.append(rec)
    return rec
