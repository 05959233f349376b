"""Mixed precision: the single-precision checked re-factorization and
iterative refinement in double (gblu_refactorize_f32, gblu_solve_refined)
reach the double-precision backward error, agree with the oracle's solution,
and fall back to the double-precision path when refinement cannot help.
Pivot decisions are double precision: a pivot that single precision cannot
place clearly on one side of the threshold sends the step to the
double-precision re-factorization, whose check and restart set the pivot
sequence."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import oracle as O
from paper_2411_14082_gb300 import gblu, inputs

pytestmark = pytest.mark.gpu

DEV = 0


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(f"cuda:{DEV}")


def forward_gap_bound(n, Ap, Ai, Ax, x, xo, b):
    """x - xo = A^{-1} (r(xo) - r(x)), so |x - xo|inf <= |A^{-1}|inf (|r(x)|inf + |r(xo)|inf);
    twice that leaves room for rounding in the residuals and the inverse."""
    A = sp.csc_matrix((Ax, Ai, Ap), shape=(n, n))
    ainv = np.abs(np.linalg.inv(A.toarray())).sum(axis=1).max()
    r = np.abs(b - A @ x).max() + np.abs(b - A @ xo).max()
    return 2.0 * ainv * r


def setup(ckt):
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, Q)
    s.factorize(dev(Ax))
    return s, n, Ap, Ai, Ax, Q


@pytest.mark.parametrize("case", ["small_mna", "mesh"])
def test_refinement_reaches_double_precision(case):
    ckt = inputs.workload_small() if case == "small_mna" else inputs.rc_mesh3d(24, 24, 4, seed=5, n_fet=60)
    s, n, Ap, Ai, Ax, Q = setup(ckt)
    rng = np.random.default_rng(3)
    lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    for it in range(3):
        ckt = inputs.perturb_elements(ckt, rng) if case == "small_mna" else inputs.redraw_transistors(ckt, rng)
        Ax = ckt.values()
        b = inputs.rhs(n, rng)
        lu = O.refactorize(lu, Ap, Ai, Ax)
        failed = s.refactorize_f32(dev(Ax))
        x, iters, berr = s.solve_refined(dev(Ax), dev(b), tol=1e-12)
        xh = x.cpu().numpy()
        assert berr <= 1e-12
        assert O.residual(n, Ap, Ai, Ax, xh, b) <= 1e-12
        xo = O.solve(lu, b)
        assert np.abs(xh - xo).max() <= forward_gap_bound(n, Ap, Ai, Ax, xh, xo, b)
        if not failed:
            assert 0 <= iters <= 5


def test_unreachable_tolerance_falls_back_to_double():
    ckt = inputs.rc_mesh3d(24, 24, 4, seed=5, n_fet=60)
    s, n, Ap, Ai, Ax, Q = setup(ckt)
    b = inputs.rhs(n, np.random.default_rng(4))
    assert not s.refactorize_f32(dev(Ax))
    x, iters, berr = s.solve_refined(dev(Ax), dev(b), tol=0.0, max_iter=3)
    assert iters == -1
    # the fallback is the double-precision path itself
    s2 = gblu.Solver(DEV)
    s2.analyze(n, Ap, Ai, Q)
    s2.factorize(dev(Ax))
    s2.refactorize(dev(Ax))
    x2 = s2.solve(dev(b))
    assert torch.equal(x, x2)
    assert berr <= 1e-12


def test_failed_single_precision_check_falls_back():
    ckt = inputs.workload_small()
    s, n, Ap, Ai, Ax, Q = setup(ckt)
    lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    k = n // 2
    while True:
        c = Q[k]
        rows = Ai[Ap[c]:Ap[c + 1]]
        hit = np.nonzero(rows == lu.piv[k])[0]
        if len(hit) and lu.Lp[k + 1] > lu.Lp[k]:
            break
        k += 1
    Ax2 = Ax.copy()
    Ax2[Ap[c] + hit[0]] -= lu.Ux[lu.Up[k + 1] - 1] * (1.0 - 1e-9)
    assert O.refactorize(lu, Ap, Ai, Ax2).n_rejected > 0
    assert s.refactorize_f32(dev(Ax2))
    b = inputs.rhs(n, np.random.default_rng(5))
    x, iters, berr = s.solve_refined(dev(Ax2), dev(b))
    assert iters == -1 and berr <= 1e-12
    assert O.residual(n, Ap, Ai, Ax2, x.cpu().numpy(), b) <= 1e-12


def test_ill_conditioned_mesh_reaches_tolerance_or_falls_back():
    """Conductances log-uniform in [1e-9, 1e4] S: single precision may not
    carry the refinement; either way the answer meets the tolerance."""
    ckt = inputs.rc_mesh3d(24, 24, 4, seed=6, n_fet=60, g_range=(1e-9, 1e4))
    s, n, Ap, Ai, Ax, Q = setup(ckt)
    rng = np.random.default_rng(12)
    lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    outcomes = set()
    for it in range(3):
        ckt = inputs.redraw_transistors(ckt, rng)
        Ax = ckt.values()
        b = inputs.rhs(n, rng)
        lu = O.refactorize(lu, Ap, Ai, Ax)
        s.refactorize_f32(dev(Ax))
        x, iters, berr = s.solve_refined(dev(Ax), dev(b), tol=1e-12, max_iter=10)
        outcomes.add(iters < 0)
        xh = x.cpu().numpy()
        assert berr <= 1e-12 and O.residual(n, Ap, Ai, Ax, xh, b) <= 1e-12
        xo = O.solve(lu, b)
        assert np.abs(xh - xo).max() <= forward_gap_bound(n, Ap, Ai, Ax, xh, xo, b)


@pytest.mark.parametrize("side", ["fails_in_double", "passes_in_double"])
def test_pivot_decision_near_the_threshold_is_taken_in_double(side):
    """One pivot of a mesh is set to eps * m * (1 -/+ 1e-6): the double
    check fails (passes) by a relative 1e-6, far below what single precision
    resolves there.  The single-precision pass cannot certify the pivot and
    reports a failed check; the refined solve then runs the double-precision
    re-factorization, and the handle ends with the pivot sequence that the
    oracle (and a double-precision handle) choose."""
    ckt = inputs.rc_mesh3d(24, 24, 4, seed=5, n_fet=60)
    s, n, Ap, Ai, Ax, Q = setup(ckt)
    lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    k = (2 * n) // 3
    c, pk = Q[k], lu.piv[k]
    rows = Ai[Ap[c]:Ap[c + 1]]
    slot = Ap[c] + int(np.nonzero(rows == pk)[0][0])
    d = lu.Ux[lu.Up[k + 1] - 1]
    m = abs(d) * np.abs(lu.Lx[lu.Lp[k]:lu.Lp[k + 1]]).max()
    t = np.sign(d) * 1e-3 * m * (1 - 1e-6 if side == "fails_in_double" else 1 + 1e-6)
    Ax2 = Ax.copy()
    Ax2[slot] += t - d
    ref = O.refactorize(lu, Ap, Ai, Ax2)
    assert ref.status == O.OK
    assert (ref.n_rejected > 0) == (side == "fails_in_double")
    assert s.refactorize_f32(dev(Ax2))
    b = inputs.rhs(n, np.random.default_rng(9))
    x, iters, berr = s.solve_refined(dev(Ax2), dev(b), tol=1e-12)
    assert iters == -1 and berr <= 1e-12
    piv = s.export_factors()["piv"]
    assert np.array_equal(piv, ref.piv)
    s64 = gblu.Solver(DEV)
    s64.analyze(n, Ap, Ai, Q)
    s64.factorize(dev(Ax))
    _, rep = s64.refactorize(dev(Ax2))
    assert rep == (side == "fails_in_double")
    assert np.array_equal(s64.export_factors()["piv"], piv)
    assert O.residual(n, Ap, Ai, Ax2, x.cpu().numpy(), b) <= 1e-12


def test_clear_pivots_keep_single_precision():
    """On the mesh every pivot clears the threshold by far more than the
    single-precision error estimate: the single-precision factors are used."""
    ckt = inputs.rc_mesh3d(24, 24, 4, seed=5, n_fet=60)
    s, n, Ap, Ai, Ax, Q = setup(ckt)
    rng = np.random.default_rng(10)
    for it in range(3):
        Ax = inputs.redraw_transistors(ckt, rng).values()
        assert not s.refactorize_f32(dev(Ax))
        b = inputs.rhs(n, rng)
        x, iters, berr = s.solve_refined(dev(Ax), dev(b), tol=1e-12)
        assert 0 <= iters <= 5 and berr <= 1e-12
