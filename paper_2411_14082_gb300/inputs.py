"""Seeded synthetic circuit matrices (modified nodal analysis, MNA).

The paper measures on SuiteSparse circuit matrices, in-house SPICE circuits
and the ibmpg power grids (Section VI); none of them is available here, so
these generators build matrices of the same kind: nodal conductance
matrices of resistor/RC grids with long-range couplings, transistor
transconductance stamps and voltage-source branch rows whose diagonal is
structurally zero (so that the factorization has to pivot).

This module is shared by the tests, the benchmark and the oracle-side
checks.  It holds no arithmetic of the LU method itself: it only stamps
circuit elements into a CSC matrix with a fixed sparsity pattern, draws
value perturbations and right-hand sides, and offers a geometric nested
dissection ordering computed from the grid coordinates (a pre-processing
input, Section III-A, not part of the factorization).

Layout of every matrix: CSC, ``indptr`` int32[n+1], ``indices`` int32[nnz]
(rows sorted inside each column, no duplicates), ``data`` float64[nnz].
The pattern is a function of the circuit topology only, so value updates
keep every slot (an entry that sums to 0.0 stays stored).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 20241121


@dataclasses.dataclass
class Circuit:
    """A linear(ised) circuit in MNA form.

    Unknowns 0..n_nodes-1 are node voltages, n_nodes..n-1 are branch
    currents of grounded voltage sources.
    """

    n_nodes: int
    # two-terminal conductances between node a and node b (b = -1: ground)
    res_a: np.ndarray
    res_b: np.ndarray
    res_g: np.ndarray
    # grounded shunt per node (capacitor companion C/h plus gmin)
    shunt: np.ndarray
    # voltage-controlled current sources: current gm*(v_c - v_s) from d to s
    vccs_d: np.ndarray
    vccs_c: np.ndarray
    vccs_s: np.ndarray
    vccs_gm: np.ndarray
    # grounded voltage sources at node vsrc_node; branch unknown n_nodes + i
    vsrc_node: np.ndarray
    # grid geometry (nx, ny, nz) of the node numbering, or None
    grid: tuple | None = None
    # nodes outside the grid (border rails), appended after the grid nodes
    n_extra_nodes: int = 0

    _pattern: tuple | None = dataclasses.field(default=None, repr=False)

    @property
    def n(self) -> int:
        return self.n_nodes + len(self.vsrc_node)

    # ------------------------------------------------------------------
    def _contributions(self):
        """(row, col, value) triplets of every stamp, in a fixed order."""
        rows, cols, vals = [], [], []

        a, b, g = self.res_a, self.res_b, self.res_g
        both = b >= 0
        rows += [a, b[both], a[both], b[both]]
        cols += [a, b[both], b[both], a[both]]
        vals += [g, g[both], -g[both], -g[both]]

        idx = np.arange(self.n_nodes)
        rows.append(idx)
        cols.append(idx)
        vals.append(self.shunt)

        d, c, s, gm = self.vccs_d, self.vccs_c, self.vccs_s, self.vccs_gm
        rows += [d, d, s, s]
        cols += [c, s, c, s]
        vals += [gm, -gm, -gm, gm]

        br = self.n_nodes + np.arange(len(self.vsrc_node))
        one = np.ones(len(br))
        rows += [self.vsrc_node, br]
        cols += [br, self.vsrc_node]
        vals += [one, one]

        return (np.concatenate(rows).astype(np.int64),
                np.concatenate(cols).astype(np.int64),
                np.concatenate(vals).astype(np.float64))

    def pattern(self):
        """CSC pattern (indptr, indices) and the stamp -> slot map."""
        if self._pattern is None:
            r, c, _ = self._contributions()
            n = self.n
            key = c * n + r
            uniq, slot = np.unique(key, return_inverse=True)
            cols = (uniq // n).astype(np.int64)
            indices = (uniq % n).astype(np.int32)
            indptr = np.zeros(n + 1, dtype=np.int64)
            np.add.at(indptr, cols + 1, 1)
            indptr = np.cumsum(indptr).astype(np.int32)
            self._pattern = (indptr, indices, slot.astype(np.int64))
        return self._pattern

    def values(self) -> np.ndarray:
        """Stamped CSC values for the current element values."""
        indptr, indices, slot = self.pattern()
        _, _, v = self._contributions()
        return np.bincount(slot, weights=v, minlength=len(indices)).astype(np.float64)

    def csc(self):
        indptr, indices, _ = self.pattern()
        return self.n, indptr, indices, self.values()

    def copy(self) -> "Circuit":
        out = dataclasses.replace(self)
        for f in ("res_a", "res_b", "res_g", "shunt", "vccs_d", "vccs_c",
                  "vccs_s", "vccs_gm", "vsrc_node"):
            setattr(out, f, getattr(self, f).copy())
        out._pattern = self._pattern
        return out


# ----------------------------------------------------------------------
# element value distributions
def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def _log_normal(rng, median, sigma, size):
    return median * np.exp(rng.normal(0.0, sigma, size))


def _grid_edges(nx, ny, nz):
    """Neighbour pairs of a (nx, ny, nz) grid: in-layer x, in-layer y, vias."""
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    ex = (idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel())
    ey = (idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel())
    ez = (idx[:-1, :, :].ravel(), idx[1:, :, :].ravel())
    return ex, ey, ez


def _random_pairs(rng, n_nodes, count):
    a = rng.integers(0, n_nodes, count)
    b = rng.integers(0, n_nodes - 1, count)
    b = np.where(b >= a, b + 1, b)          # a != b
    return a, b


# ----------------------------------------------------------------------
def mna_grid2d(nx=40, ny=50, seed=BASE_SEED, g_lo=1e-6, g_hi=1e3,
               couple_frac=0.01, n_vsrc=20, gmin=1e-12) -> Circuit:
    """2D resistor grid with grounded voltage sources (small MNA case).

    4-neighbour conductances log-uniform in [g_lo, g_hi] S, ``couple_frac``
    times the edge count of extra long-range couplings drawn from the same
    distribution, and ``n_vsrc`` grounded voltage sources at distinct random
    nodes, each adding a branch row/column with a structurally zero diagonal.
    """
    rng = np.random.default_rng(seed)
    n_nodes = nx * ny
    ex, ey, _ = _grid_edges(nx, ny, 1)
    a = np.concatenate([ex[0], ey[0]])
    b = np.concatenate([ex[1], ey[1]])
    ncoup = int(round(couple_frac * len(a)))
    ca, cb = _random_pairs(rng, n_nodes, ncoup)
    a = np.concatenate([a, ca])
    b = np.concatenate([b, cb])
    g = _log_uniform(rng, g_lo, g_hi, len(a))
    vs = rng.choice(n_nodes, size=n_vsrc, replace=False)
    e = np.zeros(0, dtype=np.int64)
    return Circuit(n_nodes=n_nodes, res_a=a, res_b=b, res_g=g,
                   shunt=np.full(n_nodes, gmin),
                   vccs_d=e, vccs_c=e, vccs_s=e, vccs_gm=np.zeros(0),
                   vsrc_node=np.sort(vs).astype(np.int64), grid=(nx, ny, 1))


def rc_mesh3d(nx=200, ny=200, nz=4, seed=BASE_SEED + 1, wire_median=1.0,
              wire_sigma=0.5, via_factor=10.0, cap_median=1e-2,
              couple_frac=0.005, n_fet=2000, gm_median=1e-3, gm_sigma=1.0,
              g_range=None) -> Circuit:
    """Post-layout power-grid style RC mesh.

    In-layer wires log-normal (median ``wire_median`` S), vias
    ``via_factor`` times a drawn wire value, a grounded C/h companion on
    every node, ``couple_frac`` x edges of random long couplings and
    ``n_fet`` transistor transconductance stamps on layer 0 whose control
    and source nodes lie within two grid steps of the drain.  With
    ``g_range=(lo, hi)`` every conductance is log-uniform in that range
    instead (the ill-conditioned variant).
    """
    rng = np.random.default_rng(seed)
    n_nodes = nx * ny * nz
    ex, ey, ez = _grid_edges(nx, ny, nz)
    wa = np.concatenate([ex[0], ey[0]])
    wb = np.concatenate([ex[1], ey[1]])
    nedge = len(wa) + len(ez[0])
    ncoup = int(round(couple_frac * nedge))
    ca, cb = _random_pairs(rng, n_nodes, ncoup)
    if g_range is None:
        gw = _log_normal(rng, wire_median, wire_sigma, len(wa))
        gv = via_factor * _log_normal(rng, wire_median, wire_sigma, len(ez[0]))
        gc = _log_normal(rng, wire_median, wire_sigma, ncoup)
        shunt = _log_normal(rng, cap_median, wire_sigma, n_nodes)
    else:
        lo, hi = g_range
        gw = _log_uniform(rng, lo, hi, len(wa))
        gv = via_factor * _log_uniform(rng, lo, hi, len(ez[0]))
        gc = _log_uniform(rng, lo, hi, ncoup)
        shunt = _log_uniform(rng, lo, hi, n_nodes) * 1e-2
    a = np.concatenate([wa, ez[0], ca])
    b = np.concatenate([wb, ez[1], cb])
    g = np.concatenate([gw, gv, gc])

    # transistor stamps on layer 0: drain d, control c and source s nearby
    dx = rng.integers(2, nx - 2, n_fet)
    dy = rng.integers(2, ny - 2, n_fet)

    def near(x, y):
        ox = rng.integers(-2, 3, len(x))
        oy = rng.integers(-2, 3, len(x))
        ox[(ox == 0) & (oy == 0)] = 1       # never the drain itself
        return (y + oy) * nx + (x + ox)

    d = dy * nx + dx
    c = near(dx, dy)
    s = near(dx, dy)
    s = np.where(s == c, np.where(c == d + 1, d - 1, d + 1), s)
    gm = _log_normal(rng, gm_median, gm_sigma, n_fet)
    e = np.zeros(0, dtype=np.int64)
    return Circuit(n_nodes=n_nodes, res_a=a, res_b=b, res_g=g, shunt=shunt,
                   vccs_d=d.astype(np.int64), vccs_c=c.astype(np.int64),
                   vccs_s=s.astype(np.int64), vccs_gm=gm,
                   vsrc_node=e, grid=(nx, ny, nz))


def bordered_grid(nx=141, ny=141, n_rails=50, density=0.05,
                  seed=BASE_SEED + 2) -> Circuit:
    """2D grid plus dense-ish power/ground rails (bordered block diagonal).

    Each of the ``n_rails`` extra nodes connects to ``density`` of the grid
    nodes (one fraction for all rails, or one per rail) with log-normal
    conductances.
    """
    rng = np.random.default_rng(seed)
    n_grid = nx * ny
    ex, ey, _ = _grid_edges(nx, ny, 1)
    a = [ex[0], ey[0]]
    b = [ex[1], ey[1]]
    dens = np.broadcast_to(np.asarray(density, dtype=np.float64), (n_rails,))
    for r in range(n_rails):
        per = max(1, int(round(dens[r] * n_grid)))
        tgt = rng.choice(n_grid, size=per, replace=False)
        a.append(np.full(per, n_grid + r))
        b.append(tgt)
    a = np.concatenate(a)
    b = np.concatenate(b)
    g = _log_normal(rng, 1.0, 0.5, len(a))
    shunt = _log_normal(rng, 1e-2, 0.5, n_grid + n_rails)
    e = np.zeros(0, dtype=np.int64)
    return Circuit(n_nodes=n_grid + n_rails, res_a=a, res_b=b, res_g=g,
                   shunt=shunt, vccs_d=e, vccs_c=e, vccs_s=e,
                   vccs_gm=np.zeros(0), vsrc_node=e, grid=(nx, ny, 1),
                   n_extra_nodes=n_rails)


# ----------------------------------------------------------------------
# value changes between Newton-Raphson iterations / time steps
def perturb_elements(ckt: Circuit, rng, frac=0.05, sigma=0.3) -> Circuit:
    """Multiply ``frac`` of the two-terminal conductances by exp(N(0, sigma))."""
    out = ckt.copy()
    m = len(out.res_g)
    k = max(1, int(round(frac * m)))
    pick = rng.choice(m, size=k, replace=False)
    out.res_g[pick] *= np.exp(rng.normal(0.0, sigma, k))
    return out


def redraw_transistors(ckt: Circuit, rng, median=1e-3, sigma=1.0) -> Circuit:
    """New transconductance values for every transistor stamp (one time step)."""
    out = ckt.copy()
    out.vccs_gm = _log_normal(rng, median, sigma, len(out.vccs_gm))
    return out


def perturb_entries(data: np.ndarray, rng, frac=0.05, sigma=0.3) -> np.ndarray:
    """Multiply ``frac`` of the stored matrix entries by exp(N(0, sigma))."""
    out = data.copy()
    k = max(1, int(round(frac * len(out))))
    pick = rng.choice(len(out), size=k, replace=False)
    out[pick] *= np.exp(rng.normal(0.0, sigma, k))
    return out


def scale_values(data: np.ndarray, rng, spread=0.2) -> np.ndarray:
    """Scale every entry by exp(N(0, ln(1+spread))) (one Monte-Carlo corner)."""
    return data * np.exp(rng.normal(0.0, math.log1p(spread), len(data)))


def rhs(n, rng) -> np.ndarray:
    return rng.uniform(-1.0, 1.0, n)


# ----------------------------------------------------------------------
def random_sparse(n, density, rng, zero_diag_frac=0.0, dominance=0.0):
    """Random CSC matrix for small tests (values N(0,1), optional zero diagonals).

    The diagonal is always structurally present except for a
    ``zero_diag_frac`` share of columns, where it is left out.
    """
    mask = rng.random((n, n)) < density
    np.fill_diagonal(mask, True)
    nodiag = rng.random(n) < zero_diag_frac
    mask[nodiag, nodiag] = False
    vals = rng.normal(0.0, 1.0, (n, n))
    if dominance:
        vals[np.arange(n), np.arange(n)] += dominance * np.sign(
            vals[np.arange(n), np.arange(n)] + 1e-300)
    dense = np.where(mask, vals, 0.0)
    return dense_to_csc(dense, mask)


def dense_to_csc(dense, mask=None):
    n = dense.shape[0]
    if mask is None:
        mask = dense != 0
    indptr = np.zeros(n + 1, dtype=np.int32)
    indices, data = [], []
    for j in range(n):
        rows = np.nonzero(mask[:, j])[0]
        indices.append(rows)
        data.append(dense[rows, j])
        indptr[j + 1] = indptr[j] + len(rows)
    return (n, indptr, np.concatenate(indices).astype(np.int32),
            np.concatenate(data).astype(np.float64))


# ----------------------------------------------------------------------
# geometric nested dissection (pre-processing input, Section III-A)
def _sym_adjacency(ckt: Circuit):
    import scipy.sparse as sp
    n = ckt.n
    indptr, indices, _ = ckt.pattern()
    a = sp.csc_matrix((np.ones(len(indices)), indices, indptr), shape=(n, n))
    s = ((a + a.T) != 0).tocsr()
    s.setdiag(0)
    s.eliminate_zeros()
    return s.indptr.astype(np.int64), s.indices.astype(np.int64)


def grid_nd_order(ckt: Circuit, leaf=16) -> np.ndarray:
    """Column ordering by recursive coordinate bisection of the grid.

    Each node set is split across the axis of its largest extent; the
    middle plane is the separator and is numbered after both halves, so the
    result is a nested dissection ordering (the ordering family the paper
    prefers for mesh-like and post-layout matrices, Section III-A).  Edges
    that are not grid edges (long couplings, transistor stamps) can join
    the two halves directly; for each such edge one endpoint is moved into
    the separator (greedy vertex cover, endpoint with more crossing edges
    first), so the separator really disconnects the halves.

    Voltage-source branch unknowns come first (a minimum-degree ordering
    picks these degree-1 nodes first too, which forces pivoting on their
    zero diagonals) and border nodes without grid coordinates come last.
    """
    nx, ny, nz = ckt.grid
    n_grid = nx * ny * nz
    adj_ptr, adj = _sym_adjacency(ckt)
    idx = np.arange(n_grid)
    coord = np.stack([idx % nx, (idx // nx) % ny, idx // (nx * ny)], axis=1)
    label = np.zeros(ckt.n, dtype=np.int8)
    out = []

    def crossing_cover(left):
        """Nodes to move so that no edge joins label 1 and label 2."""
        if len(left) == 0:
            return np.zeros(0, dtype=np.int64)
        cnt = adj_ptr[left + 1] - adj_ptr[left]
        src = np.repeat(left, cnt)
        offs = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        dst = adj[np.repeat(adj_ptr[left], cnt) + offs]
        m = label[dst] == 2
        a, b = src[m], dst[m]
        if len(a) == 0:
            return np.zeros(0, dtype=np.int64)
        ends, deg = np.unique(np.concatenate([a, b]), return_counts=True)
        dmap = dict(zip(ends.tolist(), deg.tolist()))
        moved = set()
        for u, v in zip(a.tolist(), b.tolist()):
            if u in moved or v in moved:
                continue
            moved.add(u if dmap[u] >= dmap[v] else v)
        return np.fromiter(sorted(moved), dtype=np.int64, count=len(moved))

    def rec(nodes):
        if len(nodes) <= leaf:
            out.append(nodes)
            return
        c = coord[nodes]
        lo, hi = c.min(0), c.max(0)
        ax = int(np.argmax(hi - lo))
        if hi[ax] - lo[ax] < 2:
            out.append(nodes)
            return
        mid = (lo[ax] + hi[ax]) // 2
        left = nodes[c[:, ax] < mid]
        right = nodes[c[:, ax] > mid]
        sep = nodes[c[:, ax] == mid]
        label[left] = 1
        label[right] = 2
        moved = crossing_cover(left)
        label[left] = 0
        label[right] = 0
        if len(moved):
            left = left[~np.isin(left, moved)]
            right = right[~np.isin(right, moved)]
            sep = np.concatenate([sep, moved])
        rec(left)
        rec(right)
        out.append(sep)

    rec(np.arange(n_grid, dtype=np.int64))
    grid_order = np.concatenate(out)
    branches = np.arange(ckt.n_nodes, ckt.n)
    extra = np.arange(n_grid, ckt.n_nodes)
    q = np.concatenate([branches, grid_order, extra]).astype(np.int32)
    assert len(q) == ckt.n and len(np.unique(q)) == ckt.n
    return q


# ----------------------------------------------------------------------
# named workloads
def workload_small(seed=BASE_SEED):
    """40x50 MNA grid with 20 voltage sources, n = 2,020."""
    return mna_grid2d(40, 50, seed=seed)


def workload_mesh(seed=BASE_SEED + 1, nx=200, ny=200, nz=4, **kw):
    """200x200x4 post-layout RC power-grid mesh, n = 160,000."""
    return rc_mesh3d(nx, ny, nz, seed=seed, **kw)
