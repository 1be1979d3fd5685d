"""Pins of the RCM / permutation oracle."""
import numpy as np
import pytest

import synth
from oracle import reorder
from tests.conftest import read_golden


def csr_from_edges(n, edges):
    rows, cols = [], []
    for i in range(n):
        rows.append(i)
        cols.append(i)
    for a, b in edges:
        rows += [a, b]
        cols += [b, a]
    rows, cols = np.array(rows), np.array(cols)
    return synth.matrices._from_coo(n, rows, cols, np.ones(rows.size))


def golden_cases():
    out = []
    for name_n_perm, edges in read_golden("rcm_hand.txt"):
        name, n, perm = name_n_perm.split()
        e = [tuple(int(v) for v in t.split("-")) for t in edges.split()]
        out.append((name, int(n), [int(v) for v in perm.split(",")], e))
    return out


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c[0])
def test_rcm_hand_worked(case):
    name, n, perm, edges = case
    a = csr_from_edges(n, edges)
    assert reorder.rcm_py(n, a.rowptr, a.colidx).tolist() == perm
    assert reorder.rcm(n, a.rowptr, a.colidx).tolist() == perm
    assert reorder.check_cm_order(n, a.rowptr, a.colidx, np.array(perm)) == []


def test_checker_catches_a_wrong_order():
    name, n, perm, edges = golden_cases()[0]
    a = csr_from_edges(n, edges)
    bad = list(perm)
    bad[-2], bad[-3] = bad[-3], bad[-2]       # swap two children of vertex 0
    assert reorder.check_cm_order(n, a.rowptr, a.colidx, np.array(bad)) != []


@pytest.mark.parametrize("seed", range(6))
def test_python_and_c_agree_random(seed):
    a = synth.random_pattern(70, 0.04, seed, symmetric=bool(seed % 2), empty_rows=seed)
    p1 = reorder.rcm_py(a.n, a.rowptr, a.colidx)
    p2 = reorder.rcm(a.n, a.rowptr, a.colidx)
    assert np.array_equal(p1, p2)
    assert np.array_equal(np.sort(p2), np.arange(a.n))
    assert reorder.check_cm_order(a.n, a.rowptr, a.colidx, p2) == []


def test_python_and_c_agree_grid():
    a = synth.stencil_2d_5pt(12, 9, labels=synth.vectors.permutation(108, 3))
    assert np.array_equal(reorder.rcm_py(a.n, a.rowptr, a.colidx), reorder.rcm(a.n, a.rowptr, a.colidx))


def test_path_graph_bandwidth_one():
    n = 200
    lab = synth.vectors.permutation(n, 5)
    edges = [(int(lab[i]), int(lab[i + 1])) for i in range(n - 1)]
    a = csr_from_edges(n, edges)
    perm = reorder.rcm(n, a.rowptr, a.colidx)
    brp, bci, _ = reorder.permute_scipy(n, a.rowptr, a.colidx, a.vals, perm)
    assert reorder.bandwidth(n, brp, bci) == 1


def test_scrambled_grid_bandwidth():
    a = synth.stencil_2d_5pt(64, 64, labels=synth.vectors.permutation(4096, 1))
    assert reorder.bandwidth(a.n, a.rowptr, a.colidx) > 1000
    perm = reorder.rcm(a.n, a.rowptr, a.colidx)
    brp, bci, _ = reorder.permute_scipy(a.n, a.rowptr, a.colidx, a.vals, perm)
    assert reorder.bandwidth(a.n, brp, bci) <= 2 * 64


def test_bandwidth_close_to_scipy():
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    for a in (synth.stencil_3d(12, 12, 12, 7, labels=synth.vectors.permutation(1728, 3)),
              synth.stencil_3d(10, 10, 10, 27, labels=synth.vectors.permutation(1000, 3)),
              synth.fem_like(10, 4)):
        perm = reorder.rcm(a.n, a.rowptr, a.colidx)
        brp, bci, _ = reorder.permute_scipy(a.n, a.rowptr, a.colidx, a.vals, perm)
        m = sp.csr_matrix((a.vals, a.colidx, a.rowptr), shape=(a.n, a.n))
        ps = reverse_cuthill_mckee(m, symmetric_mode=True)
        s_rp, s_ci, _ = reorder.permute_scipy(a.n, a.rowptr, a.colidx, a.vals, ps)
        assert reorder.bandwidth(a.n, brp, bci) <= 1.1 * reorder.bandwidth(a.n, s_rp, s_ci)


def test_permute_routes_agree_and_match_definition():
    a = synth.random_pattern(40, 0.15, 21, empty_rows=3)
    perm = synth.vectors.permutation(40, 22).astype(np.int32)
    r1 = reorder.permute_scipy(a.n, a.rowptr, a.colidx, a.vals, perm)
    r2 = reorder.permute_loop(a.n, a.rowptr, a.colidx, a.vals, perm)
    for u, v in zip(r1, r2):
        assert np.array_equal(u, v)
    A = np.zeros((40, 40))
    for i in range(40):
        A[i, a.colidx[a.rowptr[i]:a.rowptr[i + 1]]] = a.vals[a.rowptr[i]:a.rowptr[i + 1]]
    B = np.zeros((40, 40))
    brp, bci, bv = r1
    for i in range(40):
        B[i, bci[brp[i]:brp[i + 1]]] = bv[brp[i]:brp[i + 1]]
    assert np.array_equal(B, A[np.ix_(perm, perm)])


def test_nonsymmetric_pattern_uses_union():
    # 0 -> 2 stored only one way; RCM must still see the edge {0, 2}
    n = 3
    rowptr = np.array([0, 2, 3, 4], np.int32)
    colidx = np.array([0, 2, 1, 2], np.int32)
    p = reorder.rcm_py(n, rowptr, colidx)
    assert reorder.check_cm_order(n, rowptr, colidx, p) == []
    assert p.tolist() == reorder.rcm(n, rowptr, colidx).tolist()
