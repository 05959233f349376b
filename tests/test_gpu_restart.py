"""Forced re-pivoting (the paper's general-case protocol, Section VI-A): the
check of a chosen step fails whatever its value, the restart recomputes with
pivoting (first the unfinished steps on the installed structure, checked;
then, if a pivot must move, the unfinished steps and their elimination-tree
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


@pytest.mark.parametrize("case", ["small_mna", "mesh"])
def test_genuine_repivot_goes_through_the_pivoting_kernel(case):
    """A pivot made to fail for real (its A entry scaled by 1e-9 at a step
    without dependencies): the restart's first stage meets the same failing
    check, so the pivoting kernel recomputes the restart set; the pivot moves
    and the result is the oracle's."""
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
    assert st["tail_passes"] >= 1
    f = s.export_factors()
    assert f["piv"][k] != pr
    compare_factors(f, ref, 1e-10)
    b = inputs.rhs(n, np.random.default_rng(2))
    x = s.solve(dev(b)).cpu().numpy()
    assert O.residual(n, Ap, Ai, Ax, x, b) <= 1e-12
