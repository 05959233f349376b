"""The restart's re-prediction (Section IV-C/D with the threshold rule of
Section II-A), replayed densely on the CPU against the oracle.

A round takes the LU factors of B = A(pred, Q) without row exchanges and
checks every step in order: a step whose predicted row is its preferred one
must pass the threshold rule (|x(k)| >= eps * max of the other candidates,
x(k) != 0); a step whose preferred row went elsewhere must pivot on its
largest candidate (a strict maximum).  At the first failing step k the
candidate of largest magnitude (ties to the row first in Q) is taken, and
the step that held that row takes k's row.  The claims checked here:

- the rounds end with exactly the oracle's pivots for "prefer the previous
  pivots" (Algorithm 1 with the threshold rule), so the factors are the
  oracle's;
- the first failing step moves forward every round (the steps before it
  keep their rows and values);
- the number of rounds is the number of exchanges that lead from the
  preferred rows to the oracle's rows, first differing step first.

The LU here is a dense Doolittle elimination in numpy, a different
algorithm from the oracle's sparse left-looking one; the values are chosen
so that no decision is near a tie or the threshold.
"""
import numpy as np

from oracle import oracle as O
from paper_2411_14082_gb300 import inputs
from tests.golden_io import load

EPS = 1e-3


def dense(n, Ap, Ai, Ax):
    A = np.zeros((n, n))
    for c in range(n):
        A[Ai[Ap[c]:Ap[c + 1]], c] = Ax[Ap[c]:Ap[c + 1]]
    return A


def first_failure(A, Q, pred, prefer, qinv, strict=True, eps=EPS):
    """(k, s): the first step whose check fails on B = A(pred, Q) and the
    step of the largest candidate there; (None, None) when all pass."""
    n = len(Q)
    B = A[np.ix_(pred, Q)]
    L = np.eye(n)
    U = np.zeros((n, n))
    for k in range(n):
        # left-looking column k: U(0:k, k) by forward substitution, then x
        u = B[:k, k].copy()
        for i in range(k):
            u[i] -= L[i, :i] @ u[:i]
        x = B[k:, k] - L[k:, :k] @ u
        U[:k, k] = u
        d, others = x[0], np.abs(x[1:])
        m = others.max() if len(others) else 0.0
        if pred[k] == prefer[k] or not strict:
            ok = d != 0 and abs(d) >= eps * m
        else:
            ok = abs(d) > m
        if not ok:
            mag = np.abs(x)
            best = mag.max()
            assert best > 0
            cand = [k + j for j in np.nonzero(mag == best)[0]]
            s = min(cand, key=lambda t: qinv[pred[t]])
            return k, s
        U[k, k] = d
        L[k + 1:, k] = x[1:] / d
    return None, None


def replay(A, Q, prefer, strict=True, eps=EPS):
    """The rounds from the preferred rows: (final rows, rounds)."""
    n = len(Q)
    qinv = np.empty(n, np.int64)
    qinv[Q] = np.arange(n)
    pred, last, rounds = list(prefer), -1, 0
    while True:
        k, s = first_failure(A, Q, pred, prefer, qinv, strict, eps)
        if k is None:
            return pred, rounds
        assert k > last and s > k
        pred[k], pred[s] = pred[s], pred[k]
        last, rounds = k, rounds + 1
        assert rounds <= n


def test_worked_cascade():
    """tests/golden/repredict_cascade_3x3.txt: two rounds reach the worked
    pivots [1, 2, 0]; with the threshold rule at every step the rounds
    would stop at [1, 0, 2] (row 0 passes 0.96 >= 0.1 * 1 at step 1)."""
    g = load("repredict_cascade_3x3.txt")
    n = g["n"]
    A = dense(n, g["Ap"], g["Ai"], g["Ax"])
    prefer = [int(v) for v in g["prefer"]]
    pred, rounds = replay(A, g["Q"], prefer, eps=g["eps"])
    assert pred == [int(v) for v in g["piv"]] and rounds == 2
    assert rounds == exchange_rounds(prefer, [int(v) for v in g["piv"]])
    pred, _ = replay(A, g["Q"], prefer, strict=False, eps=g["eps"])
    assert pred == [1, 0, 2]


def exchange_rounds(prefer, piv):
    pred = list(prefer)
    pos = {r: i for i, r in enumerate(pred)}
    rounds = 0
    while True:
        bad = [i for i in range(len(pred)) if pred[i] != piv[i]]
        if not bad:
            return rounds
        k = bad[0]
        r, old = piv[k], pred[k]
        m = pos[r]
        pred[k], pred[m] = r, old
        pos[r], pos[old] = k, m
        rounds += 1


def test_repredicted_pivots_are_the_oracles():
    rng = np.random.default_rng(53)
    done = multi = 0
    for trial in range(200):
        n = int(rng.integers(4, 24))
        _, Ap, Ai, Ax0 = inputs.random_sparse(n, rng.uniform(0.15, 0.45), rng, dominance=3.0)
        Q = rng.permutation(n).astype(np.int32)
        qinv = np.empty(n, np.int64)
        qinv[Q] = np.arange(n)
        lu0 = O.factorize(n, Ap, Ai, Ax0, Q, EPS)
        if lu0.status != O.OK or not np.array_equal(lu0.piv, Q):
            continue
        prefer = [int(v) for v in lu0.piv]
        # one or two preferred pivot entries made tiny: genuine failures
        Ax = Ax0.copy()
        for k in rng.choice(n, int(rng.integers(1, 3)), replace=False):
            c = Q[k]
            hit = np.nonzero(Ai[Ap[c]:Ap[c + 1]] == prefer[k])[0]
            if len(hit):
                Ax[Ap[c] + hit[0]] *= 1e-7
        ref = O.factorize(n, Ap, Ai, Ax, Q, EPS, prefer=np.array(prefer, np.int32))
        if ref.status != O.OK or ref.n_rejected == 0:
            continue
        A = dense(n, Ap, Ai, Ax)
        if np.linalg.cond(A) > 1e8:
            continue
        pred, rounds = replay(A, Q, prefer)
        assert pred == [int(v) for v in ref.piv]
        assert rounds == exchange_rounds(prefer, [int(v) for v in ref.piv])
        done += 1
        multi += rounds > 1
    assert done >= 40 and multi >= 5
