"""Seeded sparse-matrix generators (CSR, int32 indices, FP64 values).

Every generator returns a :class:`CSR` whose rows hold strictly ascending column indices.
Random draws use ``numpy.random.default_rng(seed)`` (PCG64), which gives the same stream
on every platform numpy supports, so the same seed yields the same matrix on any host.

Workload recipes (the paper's suite, Sec. 5.3 / Table 1, is replaced by these):

* ``stencil_2d_5pt``: 2-D 5-point Laplacian, 4 on the diagonal and -1 off it.
* ``stencil_3d``: 3-D 7- or 27-point stencil on a Dirichlet (non-periodic) grid, either
  Laplacian values (6 or 26 on the diagonal, -1 off it) or diagonally dominant random
  values: each undirected edge draws one off-diagonal value from U[-1, 0) that both
  triangles share, and the diagonal is 1.01 times the row's off-diagonal absolute sum
  (symmetric positive definite).
* ``fem_like``: jittered points of a cube lattice, each linked to its 12-18 nearest
  neighbours within a radius, pattern symmetrised, off-diagonals -Exp(1) per undirected
  edge, diagonal 1.01 times the row's absolute sum.
* ``random_pattern``: small random patterns (empty rows allowed) for tiny exhaustive tests.

``labels`` assigns a new index to every vertex; the generator then emits the matrix in
that numbering.  This is how "randomly permuted" inputs are produced: the permutation is
part of the input, and undoing it is the reordering step's job.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray   # int32, n + 1
    colidx: np.ndarray   # int32, nnz
    vals: np.ndarray     # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr.astype(np.int64))


def _from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    """Sort (row, col) pairs and compress rows.  Input pairs must be unique."""
    key = rows.astype(np.int64) * n + cols.astype(np.int64)
    order = np.argsort(key, kind="stable")
    rows_s = rows[order]
    counts = np.bincount(rows_s, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    return CSR(n, rowptr.astype(np.int32), cols[order].astype(np.int32),
               np.ascontiguousarray(vals[order], dtype=np.float64))


def relabel(a: CSR, labels: np.ndarray) -> CSR:
    """Emit ``a`` with vertex v renamed ``labels[v]`` (rows and columns alike)."""
    labels = np.asarray(labels, dtype=np.int64)
    rows = np.repeat(np.arange(a.n, dtype=np.int64), a.row_lengths())
    return _from_coo(a.n, labels[rows], labels[a.colidx.astype(np.int64)], a.vals)


def _grid_csr(shape: tuple[int, ...], offsets: list[tuple[int, ...]], values: str,
              seed: int | None) -> CSR:
    """Stencil matrix on a Dirichlet grid in natural (x fastest) order.

    ``offsets`` excludes the centre.  Columns come out ascending because the offsets are
    visited in ascending linear-offset order.
    """
    dims = len(shape)
    n = int(np.prod(shape))
    strides = [1]
    for s in shape[:-1]:
        strides.append(strides[-1] * s)
    coords = np.indices(shape[::-1]).reshape(dims, -1)[::-1]   # coords[d][v], x fastest
    lin_of = lambda off: sum(o * st for o, st in zip(off, strides))
    all_offs = sorted(offsets + [tuple([0] * dims)], key=lin_of)

    masks = []
    for off in all_offs:
        m = np.ones(n, dtype=bool)
        for d in range(dims):
            if off[d] != 0:
                c = coords[d] + off[d]
                m &= (c >= 0) & (c < shape[d])
        masks.append(m)
    counts = np.sum(masks, axis=0).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    colidx = np.empty(nnz, dtype=np.int32)
    vals = np.empty(nnz, dtype=np.float64)

    # One U[-1,0) draw per undirected edge: the edge (v, v+d), d > 0, owns w_d[v].
    weights = {}
    if values == "random_dd":
        rng = np.random.default_rng(seed)
        for off in all_offs:
            if lin_of(off) > 0:
                weights[lin_of(off)] = rng.uniform(-1.0, 0.0, size=n)
    elif values != "laplacian":
        raise ValueError(values)

    fill = rowptr[:-1].copy()
    diag_pos = np.empty(n, dtype=np.int64)
    offdiag_abs = np.zeros(n, dtype=np.float64)
    for off, m in zip(all_offs, masks):
        d = lin_of(off)
        v = np.nonzero(m)[0]
        pos = fill[v]
        colidx[pos] = (v + d).astype(np.int32)
        if d == 0:
            diag_pos[v] = pos
        elif values == "laplacian":
            vals[pos] = -1.0
        else:
            w = weights[d][v] if d > 0 else weights[-d][v + d]
            vals[pos] = w
            offdiag_abs[v] += np.abs(w)
        fill[v] += 1
    if values == "laplacian":
        vals[diag_pos] = float(len(offsets))
    else:
        vals[diag_pos] = 1.01 * offdiag_abs
    return CSR(n, rowptr.astype(np.int32), colidx, vals)


def stencil_2d_5pt(nx: int, ny: int, labels: np.ndarray | None = None) -> CSR:
    offs = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    a = _grid_csr((nx, ny), offs, "laplacian", None)
    return relabel(a, labels) if labels is not None else a


def stencil_3d(nx: int, ny: int, nz: int, points: int = 7, values: str = "laplacian",
               seed: int | None = None, labels: np.ndarray | None = None) -> CSR:
    if points == 7:
        offs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    elif points == 27:
        offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                if (dx, dy, dz) != (0, 0, 0)]
    else:
        raise ValueError("points must be 7 or 27")
    a = _grid_csr((nx, ny, nz), offs, values, seed)
    return relabel(a, labels) if labels is not None else a


def fem_like(side: int, seed: int, radius: float = 1.49, kmin: int = 12, kmax: int = 18,
             scramble: bool = True) -> CSR:
    """Unstructured SPD matrix on ``side**3`` jittered lattice points.

    Point p = lattice point + U[-0.25, 0.25]^3 (lattice spacing 1).  Row p links to its
    j-th nearest neighbour for j <= ``kmin``, and for ``kmin`` < j <= ``kmax`` when that
    neighbour lies within ``radius``.  The pattern is then made symmetric (union).
    With ``scramble`` the vertices get a random labelling from the same seed.
    """
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    n = side ** 3
    lattice = np.indices((side, side, side)).reshape(3, -1).T[:, ::-1].astype(np.float64)
    pts = lattice + rng.uniform(-0.25, 0.25, size=lattice.shape)
    dist, idx = cKDTree(pts).query(pts, k=kmax + 1, workers=-1)
    dist, idx = dist[:, 1:], idx[:, 1:]
    keep = (np.arange(kmax)[None, :] < kmin) | (dist <= radius)
    r = np.repeat(np.arange(n, dtype=np.int64), keep.sum(1))
    c = idx[keep].astype(np.int64)
    lo, hi = np.minimum(r, c), np.maximum(r, c)
    und = np.unique(lo * n + hi)                       # undirected edges, sorted
    ei, ej = und // n, und % n
    w = -rng.exponential(1.0, size=und.size)
    rows = np.concatenate([ei, ej])
    cols = np.concatenate([ej, ei])
    vv = np.concatenate([w, w])
    absum = np.bincount(rows, weights=np.abs(vv), minlength=n)
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vv = np.concatenate([vv, 1.01 * absum])
    if scramble:
        labels = rng.permutation(n)
        rows, cols = labels[rows], labels[cols]
    return _from_coo(n, rows, cols, vv)


def random_pattern(n: int, density: float, seed: int, symmetric: bool = False,
                   empty_rows: int = 0, integer_values: bool = False,
                   ncols: int | None = None) -> CSR:
    """Small random sparse matrix for exhaustive tests.

    ``empty_rows`` rows (chosen at random) hold no entries.  ``integer_values`` draws
    values from {-4..4}\\{0} so sums of products are exact in FP64.
    """
    rng = np.random.default_rng(seed)
    m = ncols if ncols is not None else n
    dense = rng.random((n, m)) < density
    if symmetric:
        dense = dense | dense.T
    if empty_rows:
        dead = rng.choice(n, size=min(empty_rows, n), replace=False)
        dense[dead, :] = False
        if symmetric:
            dense[:, dead] = False
    r, c = np.nonzero(dense)
    if integer_values:
        v = rng.integers(1, 5, size=r.size) * rng.choice([-1, 1], size=r.size)
        v = v.astype(np.float64)
    else:
        v = rng.standard_normal(r.size)
    if symmetric:
        dv = np.zeros((n, m))
        dv[r, c] = v
        dv = np.triu(dv) + np.triu(dv, 1).T
        v = dv[r, c]
    out = _from_coo(n, r.astype(np.int64), c.astype(np.int64), v)
    return out


def with_dense_rows(a: CSR, count: int, length: int, seed: int) -> CSR:
    """``a`` plus ``count`` coupling rows: each chosen row (and, symmetrically, its column)
    gains ``length`` random off-diagonal entries -U[0,1); every diagonal is then reset to
    1.01 x its row's off-diagonal absolute sum, so a symmetric diagonally dominant ``a``
    stays symmetric positive definite.  Irregular (arrow-like) rows of circuit and
    constraint matrices, for the long-row path."""
    rng = np.random.default_rng(seed)
    n = a.n
    rows = np.repeat(np.arange(n, dtype=np.int64), a.row_lengths())
    cols = a.colidx.astype(np.int64)
    off = rows != cols
    r, c, v = rows[off], cols[off], a.vals[off]
    hubs = rng.choice(n, size=min(count, n), replace=False)
    extra_r, extra_c, extra_v = [], [], []
    for h in hubs:
        targets = rng.choice(n, size=min(length, n - 1) + 1, replace=False)
        targets = targets[targets != h][:length]
        w = -rng.random(targets.size)
        extra_r += [np.full(targets.size, h), targets]
        extra_c += [targets, np.full(targets.size, h)]
        extra_v += [w, w]
    r = np.concatenate([r] + extra_r)
    c = np.concatenate([c] + extra_c)
    v = np.concatenate([v] + extra_v)
    # merge repeats (a hub pair drawn twice, or an entry already in a)
    key = r * n + c
    uk, inv = np.unique(key, return_inverse=True)
    vv = np.zeros(uk.size)
    np.add.at(vv, inv, v)
    r, c, v = uk // n, uk % n, vv
    diag = np.zeros(n)
    np.add.at(diag, r, np.abs(v))
    r = np.concatenate([r, np.arange(n)])
    c = np.concatenate([c, np.arange(n)])
    v = np.concatenate([v, 1.01 * diag + (diag == 0)])
    return _from_coo(n, r, c, v)


# ---------------------------------------------------------------- batched workload
_BATCH_K = (1, 2, 4, 8, 16)


def batch_specs(count: int = 64, seed: int = 6, nmin: float = 1e3, nmax: float = 1e6):
    """Specs of the batched workload: n log-uniform in [nmin, nmax], kind cycling
    7-point / 27-point / FEM, right-hand-side count cycling {1,2,4,8,16}, value dtype
    alternating FP64 / FP32."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))
    specs = []
    for i in range(count):
        kind = ("stencil7", "stencil27", "fem")[i % 3]
        side = max(4, int(round(ns[i] ** (1.0 / 3.0))))
        specs.append(dict(index=i, kind=kind, side=side, n=side ** 3, k=_BATCH_K[i % 5],
                          dtype=("f64", "f32")[i % 2], seed=1000 + i))
    return specs


def batch_matrix(spec: dict) -> CSR:
    s = spec["side"]
    if spec["kind"] == "stencil7":
        return stencil_3d(s, s, s, 7, "random_dd", spec["seed"])
    if spec["kind"] == "stencil27":
        return stencil_3d(s, s, s, 27, "random_dd", spec["seed"])
    return fem_like(s, spec["seed"], scramble=False)
