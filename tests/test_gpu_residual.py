"""The device residual (gblu_residual) against the oracle's, output by output.

Both compute [||b - A x||_inf / (||A||_inf ||x||_inf), ||b - A x||_inf,
||A||_inf, ||x||_inf].  The device sums each row of A x in a lane tree with
fused multiply-adds, the oracle column by column without fusion, so the two
agree within the rounding of a sum of m + 1 terms (m = longest row of A):

    | ||r||_gpu - ||r||_orc | <= 2 (m + 2) u max_i (|b_i| + (|A| |x|)_i)

and the same for the row sums of |A|.  ||x|| involves no arithmetic, so it
must agree exactly.  Cases: a vector x that is not a solution (so ||r|| is
of the size of |A||x| and the bound is a relative agreement of about 1e-14),
the solution x of the system (the bench's residual check), x = 0, A scaled
near the bottom of the normal range, and NaN in x or in A.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import oracle as O
from paper_2411_14082_gb300 import gblu, inputs

pytestmark = pytest.mark.gpu

DEV = 0
U_ROUND = 2.0 ** -53


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(f"cuda:{DEV}")


def solver_for(ckt):
    n, Ap, Ai, Ax = ckt.csc()
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, inputs.grid_nd_order(ckt))
    return s, n, Ap, Ai, Ax


def compare(s, n, Ap, Ai, Ax, x, b):
    g = s.residual(dev(Ax), dev(b), dev(x)).cpu().numpy()
    o = O.residual_parts(n, Ap, Ai, Ax, x, b)
    A = sp.csc_matrix((Ax, Ai, Ap), shape=(n, n))
    m = int(np.diff(A.tocsr().indptr).max())
    scale = (np.abs(b) + abs(A) @ np.abs(x)).max()
    bound_r = 2 * (m + 2) * U_ROUND * scale
    bound_a = 2 * (m + 2) * U_ROUND * o[2]
    assert g[3] == o[3], f"||x||: {g[3]} vs {o[3]}"
    assert abs(g[1] - o[1]) <= bound_r, f"||r||: {g[1]} vs {o[1]} (bound {bound_r:.3e})"
    assert abs(g[2] - o[2]) <= bound_a, f"||A||: {g[2]} vs {o[2]} (bound {bound_a:.3e})"
    if o[2] > 0 and o[3] > 0:
        # ratio = ||r|| / (||A|| ||x||): the quotient of the checked norms,
        # each side rounded twice
        lim = (bound_r + o[1] * bound_a / o[2]) / (o[2] * o[3]) * (1 + 1e-9) + 4 * U_ROUND * o[0]
        assert abs(g[0] - o[0]) <= lim, f"ratio: {g[0]} vs {o[0]} (bound {lim:.3e})"
    else:
        assert abs(g[0] - o[0]) <= bound_r
    return g, o, bound_r


@pytest.mark.parametrize("case", ["small_mna", "mesh_30x30x4"])
def test_residual_outputs_match_oracle_on_non_solutions(case):
    ckt = inputs.workload_small() if case == "small_mna" else inputs.rc_mesh3d(30, 30, 4, seed=9, n_fet=60)
    s, n, Ap, Ai, Ax = solver_for(ckt)
    rng = np.random.default_rng(5)
    for trial in range(4):
        x = rng.uniform(-1, 1, n)
        b = rng.uniform(-1, 1, n)
        g, o, bound = compare(s, n, Ap, Ai, Ax, x, b)
        # here ||r|| is of the size of |A||x|: the outputs agree to ~1e-14 relative
        assert abs(g[1] - o[1]) <= 1e-14 * o[1]
        assert abs(g[0] - o[0]) <= 1e-14 * o[0]
        assert abs(g[2] - o[2]) <= 1e-14 * o[2]


def test_residual_of_the_solution_matches_oracle():
    ckt = inputs.workload_small()
    s, n, Ap, Ai, Ax = solver_for(ckt)
    Axd = dev(Ax)
    s.factorize(Axd)
    b = inputs.rhs(n, np.random.default_rng(8))
    x = s.solve(dev(b)).cpu().numpy()
    g, o, _ = compare(s, n, Ap, Ai, Ax, x, b)
    assert g[0] <= 1e-12 and o[0] <= 1e-12


def test_residual_degenerate_cases():
    ckt = inputs.workload_small()
    s, n, Ap, Ai, Ax = solver_for(ckt)
    rng = np.random.default_rng(6)
    b = rng.uniform(-1, 1, n)
    # x = 0: the ratio is ||b|| (no division by ||x|| = 0), on both sides exactly
    g, o, _ = compare(s, n, Ap, Ai, Ax, np.zeros(n), b)
    assert g[0] == o[0] == np.abs(b).max() and g[3] == 0.0
    # A near the bottom of the normal range (||A|| ~ 1e-295)
    tiny = Ax * 1e-298
    compare(s, n, Ap, Ai, tiny, rng.uniform(-1, 1, n), b * 1e-298)
    # A = 0: the ratio is ||b||
    g, o, _ = compare(s, n, Ap, Ai, np.zeros_like(Ax), rng.uniform(-1, 1, n), b)
    assert g[2] == 0.0 and g[0] == o[0] == np.abs(b).max()


def test_residual_propagates_nan():
    """A NaN in x or in A gives a NaN ratio on both sides: the ratio then
    fails every bound instead of hiding the NaN."""
    ckt = inputs.workload_small()
    s, n, Ap, Ai, Ax = solver_for(ckt)
    rng = np.random.default_rng(7)
    b = rng.uniform(-1, 1, n)
    for pos in (0, n // 2, n - 1):
        x = rng.uniform(-1, 1, n)
        x[pos] = np.nan
        g = s.residual(dev(Ax), dev(b), dev(x)).cpu().numpy()
        o = O.residual_parts(n, Ap, Ai, Ax, x, b)
        assert np.isnan(g[0]) and np.isnan(o[0]) and np.isnan(g[3]) and np.isnan(o[3])
        A2 = Ax.copy()
        A2[pos] = np.nan
        g = s.residual(dev(A2), dev(b), dev(rng.uniform(-1, 1, n))).cpu().numpy()
        assert np.isnan(g[0]) and np.isnan(g[2])


@pytest.mark.parametrize("where", ["below_diagonal", "diagonal", "infinite"])
def test_nonfinite_values_are_reported_not_factored(where):
    """A NaN below the diagonal, a NaN pivot, or an infinite value fails the
    pivot check; the restart reports GBLU_ERR_NONFINITE instead of storing
    the value in the factors.  The handle stays usable afterwards."""
    ckt = inputs.rc_mesh3d(20, 20, 4, seed=3, n_fet=40)
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, Q)
    s.factorize(dev(Ax))
    qinv = np.empty(n, np.int64)
    qinv[Q] = np.arange(n)
    col = int(Q[n // 3])
    rows = Ai[Ap[col]:Ap[col + 1]]
    if where == "diagonal":
        slot = Ap[col] + int(np.nonzero(rows == col)[0][0])
    else:
        below = np.nonzero(qinv[rows] > qinv[col])[0]
        slot = Ap[col] + int(below[0])
    bad = Ax.copy()
    bad[slot] = np.inf if where == "infinite" else np.nan
    with pytest.raises(gblu.GbluError) as ei:
        s.refactorize(dev(bad))
    assert ei.value.code == gblu.ERR_NONFINITE
    with pytest.raises(gblu.GbluError) as ei:
        s2 = gblu.Solver(DEV)
        s2.analyze(n, Ap, Ai, Q)
        s2.factorize(dev(bad))
    assert ei.value.code == gblu.ERR_NONFINITE
    # the handle still works on finite values
    s.factorize(dev(Ax))
    rc, _ = s.refactorize(dev(Ax))
    b = inputs.rhs(n, np.random.default_rng(1))
    x = s.solve(dev(b))
    assert s.residual(dev(Ax), dev(b), x).cpu().numpy()[0] <= 1e-12
