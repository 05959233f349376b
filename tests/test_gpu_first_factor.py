"""First factorization (Algorithm 1 with the threshold rule and the diagonal
as the preferred row) in speculative passes against the same factorization
that waits on every earlier unfinished step in order, and (the default) on
the predicted structure: the checked re-factorization kernel computes every
column there; at the first failing check the threshold rule's row is
exchanged with the row of the step that held it and the structure is
predicted again (first_mode 3), and when that gives up the pivoting kernel
computes every step (first_mode 2).

The two give the same dependencies in the same ascending order, so their
factors are bit-for-bit equal; both equal the oracle within the parity
tolerance.  The pass count follows from where the diagonal prediction
fails: one pass when every step pivots on its diagonal row; when a few
steps leave it, one more speculative pass from each such step; when many
steps leave it, a second pass that waits in order.  With more than four
absent or zero diagonal entries in A there is no speculation: one pass
that waits in order.
"""
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


def factor(n, Ap, Ai, Ax, Q, speculate):
    s = gblu.Solver(DEV, speculate_first=speculate)
    s.analyze(n, Ap, Ai, Q)
    s.factorize(dev(Ax))
    return s.export_factors(), s.stats()


def zero_diagonals(n, Ap, Ai, Ax, Q):
    """Steps whose diagonal entry A(Q[k], Q[k]) is absent or zero."""
    cnt = 0
    for c in Q:
        rows = Ai[Ap[c]:Ap[c + 1]]
        hit = np.nonzero(rows == c)[0]
        cnt += not (len(hit) and Ax[Ap[c] + hit[0]] != 0.0)
    return cnt


def same_factors(f, g):
    for key in ("piv", "Lp", "Li", "Lx", "Up", "Ui", "Ux"):
        assert np.array_equal(f[key], g[key]), key


def structure_path_taken(n, Ap, Ai, Ax, Q):
    """The library's rule for the predicted structure: every diagonal entry
    present and nonzero, at most 2% of the off-diagonal entries without
    their transposed entry."""
    if zero_diagonals(n, Ap, Ai, Ax, Q):
        return False
    cols = np.repeat(np.arange(n), np.diff(np.asarray(Ap, np.int64)))
    off = [(int(r), int(c)) for r, c in zip(Ai, cols) if r != c]
    keys = set(off)
    miss = sum((c, r) not in keys for r, c in off)
    return miss * 50 <= len(off)


def check(n, Ap, Ai, Ax, Q, rtol=1e-10):
    lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    assert lu.status == O.OK
    moved = int(np.count_nonzero(lu.piv != Q))
    fs, ss = factor(n, Ap, Ai, Ax, Q, 1)
    fw, sw = factor(n, Ap, Ai, Ax, Q, 0)
    same_factors(fs, fw)
    compare_factors(fs, lu, rtol)
    fp, sp_ = factor(n, Ap, Ai, Ax, Q, 2)
    compare_factors(fp, lu, rtol)
    if structure_path_taken(n, Ap, Ai, Ax, Q):
        if moved == 0:
            assert sp_["first_mode"] == 1 and sp_["repredictions"] == 0
            assert sp_["tail_passes"] == 0
        else:
            assert sp_["first_mode"] in (2, 3)
            if sp_["first_mode"] == 3:
                # every round fixes at least one moved step's row
                assert 1 <= sp_["repredictions"] <= moved
    else:
        assert sp_["first_mode"] == 0
        same_factors(fp, fs)
    assert sw["tail_passes"] == 1
    if moved == 0 or zero_diagonals(n, Ap, Ai, Ax, Q) > 4:
        assert ss["tail_passes"] == 1
    else:
        assert ss["tail_passes"] >= 2
    return moved, ss["tail_passes"], sp_


def test_mesh_every_step_keeps_its_diagonal():
    ckt = inputs.rc_mesh3d(40, 40, 4, seed=7, n_fet=100)
    n, Ap, Ai, Ax = ckt.csc()
    assert structure_path_taken(n, Ap, Ai, Ax, inputs.grid_nd_order(ckt))
    moved, passes, _ = check(n, Ap, Ai, Ax, inputs.grid_nd_order(ckt))
    assert moved == 0 and passes == 1


def test_mna_grid_with_voltage_sources():
    """Branch-current rows of the 20 voltage sources have zero diagonals:
    the prediction would fail at many steps, so the run does not speculate
    and waits in order in one pass."""
    ckt = inputs.workload_small()
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    assert zero_diagonals(n, Ap, Ai, Ax, Q) > 4
    moved, passes, _ = check(n, Ap, Ai, Ax, Q)
    assert moved > 4 and passes == 1


def test_one_step_leaves_its_diagonal():
    """The diagonal entry of one step is shifted so that its updated value
    becomes 1e-9 of the unshifted one, below the threshold: that step takes
    another step's row, and that step (two moved pivots in all) takes another
    row in turn.  The steps after each of the two run again, in speculative
    passes.  On the predicted structure the two steps exchange their rows:
    one re-prediction (the failing step takes the row of the step that held
    it, which takes the failing step's row) is exactly right."""
    ckt = inputs.rc_mesh3d(40, 40, 4, seed=13, n_fet=100)
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    lu0 = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    assert np.array_equal(lu0.piv, Q)
    rng = np.random.default_rng(4)
    tried = 0
    for k in rng.permutation(np.arange(n // 4, 3 * n // 4)):
        k = int(k)
        if lu0.Lp[k + 1] - lu0.Lp[k] < 2:
            continue
        c = Q[k]
        rows = Ai[Ap[c]:Ap[c + 1]]
        hit = np.nonzero(rows == c)[0]
        if not len(hit):
            continue
        Ax2 = Ax.copy()
        Ax2[Ap[c] + hit[0]] -= (1 - 1e-9) * lu0.Ux[lu0.Up[k + 1] - 1]
        lu = O.factorize(n, Ap, Ai, Ax2, Q, 1e-3)
        tried += 1
        if lu.status != O.OK or np.count_nonzero(lu.piv != Q) != 2:
            assert tried < 20
            continue
        assert structure_path_taken(n, Ap, Ai, Ax2, Q)
        moved, passes, sp_ = check(n, Ap, Ai, Ax2, Q)
        assert moved == 2 and passes in (2, 3)
        assert sp_["first_mode"] == 3 and sp_["repredictions"] == 1
        return
    pytest.fail("no step found whose shifted diagonal swaps two pivots")


def test_random_matrices_with_zero_diagonals():
    """n up to 300 with up to 10% density: the threshold rule (eps 1e-3)
    admits L entries up to 1e3, which carry rounding differences from one
    column to the next.  Two valid update orders of the same factorization
    differ here by up to 1.8e-10 of the componentwise scale (the oracle
    against a dense right-looking LU in numpy with the oracle's pivots), so
    the oracle comparison takes 1e-9; speculative and waiting passes must
    still agree bit for bit."""
    rng = np.random.default_rng(21)
    done = 0
    for trial in range(40):
        n = int(rng.integers(20, 300))
        _, Ap, Ai, Ax = inputs.random_sparse(n, rng.uniform(0.01, 0.1), rng,
                                             zero_diag_frac=rng.uniform(0, 0.2), dominance=1.0)
        Q = rng.permutation(n).astype(np.int32)
        A = np.zeros((n, n))
        for c in range(n):
            A[Ai[Ap[c]:Ap[c + 1]], c] = Ax[Ap[c]:Ap[c + 1]]
        if np.linalg.cond(A) > 1e12:
            continue
        if O.factorize(n, Ap, Ai, Ax, Q, 1e-3).status != O.OK:
            continue
        check(n, Ap, Ai, Ax, Q, rtol=1e-9)
        done += 1
    assert done >= 10


def test_singular_matrix_is_reported_after_speculation():
    # numerically singular 3x3: column 1 is twice column 0, so step 1 has no
    # nonzero candidate
    Ap = np.array([0, 3, 6, 9])
    Ai = np.array([0, 1, 2, 0, 1, 2, 0, 1, 2])
    Ax = np.array([1.0, 2.0, 3.0, 2.0, 4.0, 6.0, 1.0, 0.0, 1.0])
    for speculate in (2, 1, 0):
        s = gblu.Solver(DEV, speculate_first=speculate)
        s.analyze(3, Ap, Ai, np.arange(3))
        with pytest.raises(gblu.GbluError) as ei:
            s.factorize(dev(Ax))
        assert ei.value.code == gblu.ERR_SINGULAR
