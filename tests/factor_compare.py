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
and asserted (<= rtol) on every column above the rounding noise floor.  The
floor is measured, not guessed: the oracle factorizes A again with every
value moved by a few units in the last place (same pivot sequence), and a
column whose own oracle result then moves by more than rtol / 100 (relative
to its norm) is sensitive at the rounding level, so two valid summation
orders can differ there by more than rtol; the strict metric is asserted on
all other columns.
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


SENSITIVE = 1e-2   # a column is at the noise floor when the oracle moves by rtol * SENSITIVE
LOG = []   # one dict per compare_factors call (printed by tests run with -s)


def compare_part(n, gp, gi, gx, op, oi, ox, scale_of):
    """Oracle entries must all be in the GPU pattern; GPU-only entries must be
    exact zeros.  Returns (max |diff| / scale over the oracle entries,
    per-column max |diff|, per-column max |oracle entry|)."""
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
    cdiff, cnorm = np.zeros(n), np.zeros(n)
    if len(ok):
        np.maximum.at(cdiff, ocols, diff)
        np.maximum.at(cnorm, ocols, np.abs(ox))
    return (float(err.max()) if len(err) else 0.0), cdiff, cnorm


def column_sensitivity(lu, seed=0):
    """Per-column relative change (L, U) of the oracle's factors when every
    value of A is moved by up to 2 units in the last place, with the same
    pivot preference; columns from the first step whose pivot then differs
    are infinitely sensitive.  None when the oracle result has no inputs."""
    from oracle import oracle as O
    if lu.inputs is None:
        return None
    Ap, Ai, Ax = lu.inputs
    rng = np.random.default_rng(seed)
    Axp = Ax * (1.0 + rng.uniform(-2.0, 2.0, len(Ax)) * 2.0 ** -53)
    lu2 = O.factorize(lu.n, Ap, Ai, Axp, lu.Q, lu.eps, prefer=lu.piv, lib=lu._lib)
    n = lu.n
    sl, su = np.full(n, np.inf), np.full(n, np.inf)
    if lu2.status != O.OK:
        return sl, su
    same = lu2.piv == lu.piv
    k0 = n if same.all() else int(np.argmin(same))
    for part, out in (("L", sl), ("U", su)):
        p, x, x2 = getattr(lu, part + "p"), getattr(lu, part + "x"), getattr(lu2, part + "x")
        if not np.array_equal(p, getattr(lu2, part + "p")):
            return sl, su
        cols = np.repeat(np.arange(n), np.diff(np.asarray(p, np.int64)))
        d, nm = np.zeros(n), np.zeros(n)
        np.maximum.at(d, cols, np.abs(x - x2))
        np.maximum.at(nm, cols, np.abs(x))
        rel = np.where(nm > 0, d / np.where(nm > 0, nm, 1.0), 0.0)
        out[:k0] = rel[:k0]
    return sl, su


def strict_columns(cdiff, cnorm, sens, rtol):
    """Strict per-column errors; columns above the noise floor are asserted."""
    has = cnorm > 0
    rel = np.where(has, cdiff / np.where(has, cnorm, 1.0), 0.0)
    above = has if sens is None else has & (sens <= SENSITIVE * rtol)
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

    el, ldiff, lnorm = compare_part(n, f["Lp"], f["Li"], f["Lx"], lu.Lp, lu.Li, lu.Lx,
                                    lambda keys, cols: np.maximum(m_at(keys), xcol[cols]) / udiag[cols])
    eu, udiff, unorm = compare_part(n, f["Up"], f["Ui"], f["Ux"], lu.Up, lu.Ui, lu.Ux,
                                    lambda keys, cols: np.maximum(m_at(keys), xcol[cols]))
    assert el <= rtol and eu <= rtol, f"factor mismatch: L {el:.3e}, U {eu:.3e} (tol {rtol})"
    sens = column_sensitivity(lu)
    sl = strict_columns(ldiff, lnorm, None if sens is None else sens[0], rtol)
    su = strict_columns(udiff, unorm, None if sens is None else sens[1], rtol)
    rec = dict(n=n, componentwise=max(el, eu), strict_above_floor=max(sl[0], su[0]),
               strict_all=max(sl[3], su[3]), l_cols_checked=sl[1], l_cols=sl[2],
               u_cols_checked=su[1], u_cols=su[2])
    LOG.append(rec)
    return rec
