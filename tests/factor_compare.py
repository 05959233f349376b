"""Element-wise comparison of exported GPU factors with oracle factors."""
import numpy as np


def _keys(p, i, n):
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(np.asarray(p, dtype=np.int64)))
    return cols * n + np.asarray(i, dtype=np.int64), cols


def compare_part(n, gp, gi, gx, op, oi, ox, rtol):
    """Oracle entries must all be in the GPU pattern with values within
    rtol * (column inf-norm of the oracle); GPU-only entries must be 0.0
    (structural zeros of a superset pattern).  Returns the max relative error."""
    gk, _ = _keys(gp, gi, n)
    ok, ocols = _keys(op, oi, n)
    pos = np.searchsorted(gk, ok)
    assert np.all(pos < len(gk)) and np.array_equal(gk[np.minimum(pos, len(gk) - 1)], ok), \
        "an oracle entry is missing from the GPU pattern"
    extra = np.ones(len(gk), dtype=bool)
    extra[pos] = False
    assert np.all(gx[extra] == 0.0), "GPU-only pattern entries must be exact zeros"
    colnorm = np.zeros(n)
    np.maximum.at(colnorm, ocols, np.abs(ox))
    scale = np.where(colnorm[ocols] > 0, colnorm[ocols], 1.0)
    err = np.abs(gx[pos] - ox) / scale
    return float(err.max()) if len(err) else 0.0


def compare_factors(f, lu, rtol=1e-10):
    """Same column order, same pivot sequence, L and U within rtol per column."""
    n = lu.n
    assert np.array_equal(f["q"], lu.Q)
    assert np.array_equal(f["piv"], lu.piv), \
        f"pivot sequences differ at steps {np.nonzero(f['piv'] != lu.piv)[0][:10]}"
    el = compare_part(n, f["Lp"], f["Li"], f["Lx"], lu.Lp, lu.Li, lu.Lx, rtol)
    eu = compare_part(n, f["Up"], f["Ui"], f["Ux"], lu.Up, lu.Ui, lu.Ux, rtol)
    assert el <= rtol and eu <= rtol, f"factor mismatch: L {el:.3e}, U {eu:.3e} (tol {rtol})"
    return max(el, eu)
