"""The seeded generators produce the workloads' stated structure (closed-form nnz counts,
symmetric patterns and values, regular row lengths)."""
import numpy as np
import scipy.sparse as sp

import synth


def _sp(a):
    return sp.csr_matrix((a.vals, a.colidx, a.rowptr), shape=(a.n, a.n))


def test_stencil_nnz_closed_forms():
    a = synth.stencil_2d_5pt(64, 64)
    assert (a.n, a.nnz) == (4096, 5 * 4096 - 2 * 64 - 2 * 64) == (4096, 20224)
    b = synth.stencil_3d(10, 9, 8, 7)
    assert b.nnz == 7 * 720 - 2 * (10 * 9 + 9 * 8 + 10 * 8)
    c = synth.stencil_3d(10, 9, 8, 27)
    assert c.nnz == (3 * 10 - 2) * (3 * 9 - 2) * (3 * 8 - 2)


def test_rows_sorted_and_unique():
    for a in (synth.stencil_3d(5, 6, 7, 27, "random_dd", 3), synth.fem_like(8, 4),
              synth.random_pattern(40, 0.2, 1, empty_rows=5)):
        for i in range(a.n):
            row = a.colidx[a.rowptr[i]:a.rowptr[i + 1]]
            assert np.all(np.diff(row) > 0)
        assert a.rowptr.dtype == np.int32 and a.colidx.dtype == np.int32


def test_random_dd_symmetric_and_dominant():
    for a in (synth.stencil_3d(6, 5, 4, 27, "random_dd", 3), synth.stencil_3d(6, 5, 4, 7, "random_dd", 3),
              synth.fem_like(8, 4)):
        m = _sp(a)
        assert abs(m - m.T).max() == 0.0
        d = m.diagonal()
        off = np.asarray(abs(m).sum(1)).ravel() - np.abs(d)
        assert np.allclose(d, 1.01 * off)
        offv = m - sp.diags(d)
        assert offv.max() <= 0.0


def test_stencil_values_in_range():
    a = synth.stencil_3d(6, 6, 6, 7, "random_dd", 11)
    m = _sp(a) - sp.diags(_sp(a).diagonal())
    v = m.data[m.data != 0]
    assert v.min() >= -1.0 and v.max() < 0.0


def test_relabel_is_a_symmetric_permutation():
    a = synth.stencil_2d_5pt(8, 8)
    lab = synth.vectors.permutation(a.n, 1)
    b = synth.relabel(a, lab)
    A, B = _sp(a).toarray(), _sp(b).toarray()
    assert np.array_equal(B[np.ix_(lab, lab)], A)


def test_fem_like_regular():
    a = synth.fem_like(12, 4)
    lens = a.row_lengths()
    assert lens.min() >= 13          # >= 12 neighbours plus the diagonal
    assert lens.var() <= 10.0        # "regular" in the sense of Sec. 5.3


def test_seeds_reproduce():
    a1 = synth.stencil_3d(5, 5, 5, 27, "random_dd", 3)
    a2 = synth.stencil_3d(5, 5, 5, 27, "random_dd", 3)
    assert np.array_equal(a1.vals, a2.vals)
    assert np.array_equal(synth.uniform_vector(10, 2), synth.uniform_vector(10, 2))


def test_batch_specs():
    specs = synth.batch_specs()
    assert len(specs) == 64
    ns = np.array([s["n"] for s in specs])
    assert ns.min() >= 4 ** 3 and ns.max() <= 1.1e6
    assert {s["k"] for s in specs} == {1, 2, 4, 8, 16}
