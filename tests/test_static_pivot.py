"""Static pivoting and scaling (gblu_static_pivot, host code): the
permutation reaches the maximum diagonal product of the oracle (an
assignment solver on the definition) and of brute force, the scalings have
their defining properties, and the permuted pattern is P A."""
import numpy as np
import pytest

from oracle import static_pivot as SP
from paper_2411_14082_gb300 import gblu, inputs


def random_csc(n, density, rng, zero_diag=0.3):
    A = np.where(rng.random((n, n)) < density, rng.standard_normal((n, n)) * np.exp(rng.uniform(-8, 8, (n, n))), 0.0)
    zd = rng.random(n) < zero_diag                       # some zero diagonal entries
    A[np.arange(n)[zd], np.arange(n)[zd]] = 0.0
    A[rng.permutation(n), np.arange(n)] += 3.0 + rng.random(n)   # a perfect matching exists
    Ap = np.zeros(n + 1, np.int32)
    Ai, Ax = [], []
    for j in range(n):
        r = np.nonzero(A[:, j])[0]
        Ai.extend(r)
        Ax.extend(A[r, j])
        Ap[j + 1] = len(Ai)
    return Ap, np.array(Ai, np.int32), np.array(Ax)


@pytest.mark.parametrize("n", [1, 2, 5, 7])
def test_brute_force_pins_the_oracle_and_the_library(n):
    rng = np.random.default_rng(100 + n)
    for _ in range(5):
        Ap, Ai, Ax = random_csc(n, 0.5, rng)
        _, best = SP.brute_force_matching(n, Ap, Ai, Ax)
        _, orc = SP.max_product_matching(n, Ap, Ai, Ax)
        match, dr, dc = gblu.static_pivot(n, Ap, Ai, Ax)
        A = SP._dense(n, Ap, Ai, Ax)
        got = float(np.log(np.abs(A[match, np.arange(n)])).sum())
        assert abs(orc - best) <= 1e-9 * max(1.0, abs(best))
        assert abs(got - best) <= 1e-9 * max(1.0, abs(best))


@pytest.mark.parametrize("n,density", [(17, 0.2), (60, 0.08), (150, 0.03)])
def test_optimal_product_and_scaling_properties(n, density):
    rng = np.random.default_rng(n)
    for _ in range(3):
        Ap, Ai, Ax = random_csc(n, density, rng)
        match, dr, dc = gblu.static_pivot(n, Ap, Ai, Ax)
        assert sorted(match.tolist()) == list(range(n))
        _, orc = SP.max_product_matching(n, Ap, Ai, Ax)
        A = SP._dense(n, Ap, Ai, Ax)
        got = float(np.log(np.abs(A[match, np.arange(n)])).sum())
        assert abs(got - orc) <= 1e-9 * max(1.0, abs(orc))
        ok_bound, ok_diag = SP.check_scaling(n, Ap, Ai, Ax, match, dr, dc, tol=1e-10)
        assert ok_bound and ok_diag


def test_mna_matrix_gets_a_zero_free_diagonal():
    """Voltage-source branch rows have zero diagonals; the matching moves a
    nonzero onto every diagonal position."""
    ckt = inputs.workload_small()
    n, Ap, Ai, Ax = ckt.csc()
    A = SP._dense(n, Ap, Ai, Ax)
    assert np.any(np.diag(A) == 0.0)
    match, dr, dc = gblu.static_pivot(n, Ap, Ai, Ax)
    assert np.all(A[match, np.arange(n)] != 0.0)
    _, orc = SP.max_product_matching(n, Ap, Ai, Ax)
    got = float(np.log(np.abs(A[match, np.arange(n)])).sum())
    assert abs(got - orc) <= 1e-9 * abs(orc)
    ok_bound, ok_diag = SP.check_scaling(n, Ap, Ai, Ax, match, dr, dc, tol=1e-10)
    assert ok_bound and ok_diag


def test_permuted_pattern_is_PA():
    rng = np.random.default_rng(5)
    n = 40
    Ap, Ai, Ax = random_csc(n, 0.1, rng)
    match, _, _ = gblu.static_pivot(n, Ap, Ai, Ax)
    Ai2, src = gblu.permute_rows(n, Ap, Ai, match)
    A = SP._dense(n, Ap, Ai, Ax)
    B = SP._dense(n, Ap, Ai2, Ax[src])
    assert np.array_equal(B, A[match, :])
    for j in range(n):
        assert np.all(np.diff(Ai2[Ap[j]:Ap[j + 1]]) > 0)


def test_structurally_singular_is_reported():
    # two columns that can only use the same row
    Ap = np.array([0, 1, 2, 4], np.int32)
    Ai = np.array([0, 0, 1, 2], np.int32)
    Ax = np.array([1.0, 2.0, 3.0, 4.0])
    assert SP.max_product_matching(3, Ap, Ai, Ax)[0] is None
    with pytest.raises(gblu.GbluError) as e:
        gblu.static_pivot(3, Ap, Ai, Ax)
    assert e.value.code == gblu.ERR_SINGULAR
