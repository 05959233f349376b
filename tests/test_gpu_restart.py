"""Forced re-pivoting (the paper's general-case protocol, Section VI-A): the
check of a chosen step fails whatever its value, the restart recomputes the
unfinished steps and their elimination-tree ancestors with pivoting, and the
result is the oracle's factorization that prefers the previous pivots."""
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
