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
and asserted (<= rtol) on every column above the rounding noise floor.  A
column is at the floor, where two valid summation orders can differ by more
than rtol, when one of its dependencies is at the floor (it inherits that
rounding-level error through L(:,j) U(j,k)) or when
  * cancellation took more than three digits from it: the largest |L||U|
    magnitude summed into one of its entries exceeds 1e3 times the column's
    norm (for L: its norm times |U(k,k)|, and the pivot's own ratio
    (|L||U|)(k,k) / |U(k,k)|, since L(:,k) is divided by the pivot), or
  * it is sensitive to rounding-level changes of A: the oracle factorizes A
    again with every value moved by up to two units in the last place (same
    pivot sequence), and the column moves by more than rtol / 100.
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
CANCEL = 1e3       # ... or when cancellation took more than three digits from it
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


def at_floor(lu, l_ratio, u_ratio, sens, rtol):
    """Columns at the noise floor: cancellation or rounding sensitivity of
    their own, or a dependency (a U row j of column k) at the floor, whose
    rounding-level error the column inherits through L(:,j) U(j,k)."""
    n = lu.n
    own = (l_ratio > CANCEL) | (u_ratio > CANCEL)
    if sens is not None:
        own |= (sens[0] > SENSITIVE * rtol) | (sens[1] > SENSITIVE * rtol)
    bad = own.copy()
    Up = np.asarray(lu.Up, np.int64)
    for k in range(n):
        if not bad[k]:
            deps = lu.Ui[Up[k]:Up[k + 1] - 1]
            bad[k] = bool(bad[deps].any()) if len(deps) else False
    return bad


def strict_columns(cdiff, cnorm, floor, rtol):
    """Strict per-column errors; columns above the noise floor are asserted."""
    has = cnorm > 0
    rel = np.where(has, cdiff / np.where(has, cnorm, 1.0), 0.0)
    above = has & ~floor
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
    # cancellation ratio of each column: the largest |L||U| magnitude summed
    # into an entry over the column's norm (for L also the pivot's own ratio,
    # since L(:,k) is divided by it)
    lk, lcols = _keys(lu.Lp, lu.Li, n)
    uk, ucols = _keys(lu.Up, lu.Ui, n)
    lmag, umag = np.zeros(n), np.zeros(n)
    if len(lk):
        np.maximum.at(lmag, lcols, m_at(lk))
    if len(uk):
        np.maximum.at(umag, ucols, m_at(uk))
    diag = np.arange(n, dtype=np.int64)
    piv_ratio = m_at(diag * n + diag) / np.where(udiag > 0, udiag, 1.0)
    l_ratio = np.maximum(piv_ratio, lmag / np.where(lnorm > 0, udiag * lnorm, 1.0))
    u_ratio = umag / np.where(unorm > 0, unorm, 1.0)
    assert el <= rtol and eu <= rtol, f"factor mismatch: L {el:.3e}, U {eu:.3e} (tol {rtol})"
    sens = column_sensitivity(lu)
    floor = at_floor(lu, l_ratio, u_ratio, sens, rtol)
    sl = strict_columns(ldiff, lnorm, floor, rtol)
    su = strict_columns(udiff, unorm, floor, rtol)
    rec = dict(n=n, componentwise=max(el, eu), strict_above_floor=max(sl[0], su[0]),
               strict_all=max(sl[3], su[3]), l_cols_checked=sl[1], l_cols=sl[2],
               u_cols_checked=su[1], u_cols=su[2])
    LOG.append(rec)
    return rec
