"""CPU checks of the seeded synthetic inputs (the stand-ins for the paper's
circuit matrices): sizes, structure and value ranges of each workload as
the input recipe states them, and determinism."""
import numpy as np
import scipy.sparse as sp

from paper_2411_14082_gb300 import inputs


def matrix(ckt):
    n, Ap, Ai, Ax = ckt.csc()
    return n, sp.csc_matrix((Ax, Ai, Ap), shape=(n, n))


def test_small_mna_grid():
    """40x50 grid, 20 grounded voltage sources as branch rows and columns
    with zero diagonals, conductances log-uniform in [1e-6, 1e3] S."""
    ckt = inputs.workload_small()
    n, A = matrix(ckt)
    assert n == 2020 and ckt.n_nodes == 2000 and len(ckt.vsrc_node) == 20
    d = A.diagonal()
    assert np.all(d[2000:] == 0) and np.all(d[:2000] > 0)
    S = (A != 0).astype(int)
    assert (S != S.T).nnz == 0                      # structurally symmetric
    assert 9000 < A.nnz < 11000
    assert ckt.res_g.min() >= 1e-6 and ckt.res_g.max() <= 1e3
    assert np.log10(ckt.res_g).max() - np.log10(ckt.res_g).min() > 8


def test_rc_mesh_workload():
    """200x200x4 mesh, n = 160,000; every node grounded through its
    capacitance term; 2,000 transistor stamps make the pattern unsymmetric."""
    ckt = inputs.workload_mesh()
    n, A = matrix(ckt)
    assert n == 160000 and len(ckt.vsrc_node) == 0
    assert 1.0e6 < A.nnz < 1.1e6
    assert np.all(ckt.shunt > 0)
    assert len(ckt.vccs_gm) == 2000
    S = (A != 0).astype(int)
    assert (S != S.T).nnz > 0


def test_bordered_grid():
    """141x141 grid plus 50 rails joined to 5% of the grid: n = 19,931."""
    ckt = inputs.bordered_grid()
    n, A = matrix(ckt)
    assert n == 141 * 141 + 50
    dense_cols = np.diff(A.indptr)[-50:]
    assert dense_cols.min() > 0.03 * 141 * 141


def test_generators_are_deterministic_and_perturbations_local():
    a = inputs.workload_small().csc()
    b = inputs.workload_small().csc()
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)
    ckt = inputs.workload_small()
    rng = np.random.default_rng(1)
    new = inputs.perturb_elements(ckt, rng, frac=0.05)
    changed = np.count_nonzero(new.res_g != ckt.res_g)
    assert 0.03 * len(ckt.res_g) <= changed <= 0.07 * len(ckt.res_g)
    assert np.array_equal(new.csc()[1], ckt.csc()[1])   # same pattern
