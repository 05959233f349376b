"""Forced re-pivoting (the paper's general-case protocol, Section VI-A): the
check of a chosen step fails whatever its value, the restart recomputes with
pivoting (first the unfinished steps on the installed structure, checked;
then, if a pivot must move, either re-predicted structures, on a structure
that was predicted, or the unfinished steps and their elimination-tree
ancestors in the pivoting kernel), and the result is the oracle's
factorization that prefers the previous pivots.  A genuine failure takes the
second stage."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_14082_gb300 import gblu, inputs
from tests.factor_compare import compare_factors

pytestmark = pytest.mark.gpu

DEV = 0


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(f"cuda:{DEV}")


@pytest.mark.parametrize("case", ["small_mna", "mesh"])
def test_forced_repivot_matches_oracle(case):
    ckt = inputs.workload_small() if case == "small_mna" else inputs.rc_mesh3d(24, 24, 4, seed=5, n_fet=60)
    n, Ap, Ai, Ax0 = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, Q)
    s.factorize(dev(Ax0))
    lu = O.factorize(n, Ap, Ai, Ax0, Q, 1e-3)
    rng = np.random.default_rng(8)
    for force in (0, n // 3, n - 1, int(rng.integers(0, n))):
        ckt = inputs.perturb_elements(ckt, rng) if case == "small_mna" else inputs.redraw_transistors(ckt, rng)
        Ax = ckt.values()
        lu = O.refactorize(lu, Ap, Ai, Ax)
        rc, rep = s.refactorize_forced(dev(Ax), force)
        assert rep and rc == gblu.REPIVOTED
        assert s.last_status() == gblu.REPIVOTED
        st = s.stats()
        assert st["n_restart_cols"] >= 1 and st["tail_kernel_ms"] > 0
        if lu.n_rejected == 0:
            # no pivot needs to move: the restart's first stage (the
            # unfinished columns on the installed structure, checked) suffices
            assert st["tail_passes"] == 0
        compare_factors(s.export_factors(), lu, 1e-10)
        b = inputs.rhs(n, rng)
        x = s.solve(dev(b)).cpu().numpy()
        assert O.residual(n, Ap, Ai, Ax, x, b) <= 1e-12
    # no forcing: an ordinary checked refactorization again
    rc, rep = s.refactorize_forced(dev(Ax), -1)
    assert not rep and rc == gblu.OK
    assert s.last_status() == gblu.OK
    with pytest.raises(gblu.GbluError):
        s.refactorize_forced(dev(Ax), n)


def exchange_rounds(prefer, piv):
    """Rounds of the restart's re-prediction that lead from the preferred
    rows to the rows piv that the threshold rule takes: each round finds the
    first step whose predicted row is not its row in piv, gives it that row
    and gives the step that held the row the replaced one (the exact first
    failure of the checked re-factorization, since every step before it
    already has its final row)."""
    pred = np.array(prefer, np.int64)
    pinv = np.empty(len(pred), np.int64)
    pinv[pred] = np.arange(len(pred))
    rounds = 0
    while True:
        bad = np.nonzero(pred != piv)[0]
        if not len(bad):
            return rounds
        k = int(bad[0])
        r, old = int(piv[k]), int(pred[k])
        m = int(pinv[r])
        pred[k], pred[m] = r, old
        pinv[r], pinv[old] = k, m
        rounds += 1


def scaled_leaf(Ap, Ai, Ax0, Q, lu, k):
    """A's pivot entry of step k (a step without dependencies, so the
    pivot is that entry) scaled by 1e-9: its check fails for real."""
    c, pr = int(Q[k]), int(lu.piv[k])
    slot = int(Ap[c]) + int(np.nonzero(Ai[Ap[c]:Ap[c + 1]] == pr)[0][0])
    Ax = Ax0.copy()
    Ax[slot] *= 1e-9
    return Ax


@pytest.mark.parametrize("case", ["small_mna", "mesh"])
def test_genuine_repivot_matches_oracle(case):
    """A pivot made to fail for real (its A entry scaled by 1e-9 at a step
    without dependencies): the restart's first stage meets the same failing
    check, so a pivot moves.  The MNA grid's structure came from the
    pivoting kernel (zero diagonals), so its restart set goes through the
    pivoting kernel; the mesh's structure is a prediction, so the restart
    predicts it again, in as many rounds as the oracle's pivots imply.
    Either way the result is the oracle's."""
    ckt = inputs.workload_small() if case == "small_mna" else inputs.rc_mesh3d(24, 24, 4, seed=5, n_fet=60)
    n, Ap, Ai, Ax0 = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, Q)
    s.factorize(dev(Ax0))
    f0 = s.export_factors()
    lu = O.factorize(n, Ap, Ai, Ax0, Q, 1e-3)
    leaves = np.nonzero((np.diff(f0["Up"]) == 1) & (np.diff(f0["Lp"]) > 0))[0]
    for k in leaves[len(leaves) // 2:][:20]:   # a leaf where the scaled pivot really fails
        k = int(k)
        c, pr = int(Q[k]), int(f0["piv"][k])
        slot = int(Ap[c]) + int(np.nonzero(Ai[Ap[c]:Ap[c + 1]] == pr)[0][0])
        Ax = Ax0.copy()
        Ax[slot] *= 1e-9
        ref = O.refactorize(lu, Ap, Ai, Ax)
        if ref.status == O.OK and ref.n_rejected > 0:
            break
    assert ref.n_rejected > 0
    rc, rep = s.refactorize(dev(Ax))
    assert rep and rc == gblu.REPIVOTED
    st = s.stats()
    if case == "small_mna":
        assert st["tail_passes"] >= 1 and st["repredictions"] == 0
    else:
        assert st["repredictions"] == exchange_rounds(lu.piv, ref.piv)
        assert st["tail_passes"] == 0
    f = s.export_factors()
    assert f["piv"][k] != pr
    compare_factors(f, ref, 1e-10)
    b = inputs.rhs(n, np.random.default_rng(2))
    x = s.solve(dev(b)).cpu().numpy()
    assert O.residual(n, Ap, Ai, Ax, x, b) <= 1e-12


@pytest.mark.parametrize("rounds", [1, 2, 3, 4])
def test_repredicted_restart_rounds(rounds):
    """Genuine failures on a mesh whose cascades of moved pivots take one to
    four rounds of re-prediction: after the first exchange, a step whose
    preferred row went to an earlier step must pivot on its largest
    candidate (the strict check), and a wrong guess for it costs a round.
    Each restart gives the oracle's factors; the same values then
    re-factorize without a restart, bit for bit as before."""
    ckt = inputs.rc_mesh3d(24, 24, 4, seed=5, n_fet=60)
    n, Ap, Ai, Ax0 = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    lu = O.factorize(n, Ap, Ai, Ax0, Q, 1e-3)
    leaves = np.nonzero((np.diff(lu.Up) == 1) & (np.diff(lu.Lp) > 0))[0]
    for k in leaves:
        Ax = scaled_leaf(Ap, Ai, Ax0, Q, lu, int(k))
        ref = O.refactorize(lu, Ap, Ai, Ax)
        if ref.status == O.OK and exchange_rounds(lu.piv, ref.piv) == rounds:
            break
    else:
        pytest.fail(f"no leaf whose restart takes {rounds} rounds")
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, Q)
    s.factorize(dev(Ax0))
    assert s.stats()["first_mode"] == 1
    rc, rep = s.refactorize(dev(Ax))
    assert rep and rc == gblu.REPIVOTED
    st = s.stats()
    assert st["repredictions"] == rounds and st["tail_passes"] == 0
    assert st["n_repivot"] == 1
    f = s.export_factors()
    assert np.array_equal(f["piv"], ref.piv)
    compare_factors(f, ref, 1e-10)
    b = inputs.rhs(n, np.random.default_rng(rounds))
    x = s.solve(dev(b)).cpu().numpy()
    assert O.residual(n, Ap, Ai, Ax, x, b) <= 1e-12
    rc, rep = s.refactorize(dev(Ax))
    assert not rep and rc == gblu.OK
    g = s.export_factors()
    for key in ("piv", "Lp", "Li", "Lx", "Up", "Ui", "Ux"):
        assert np.array_equal(f[key], g[key]), key
