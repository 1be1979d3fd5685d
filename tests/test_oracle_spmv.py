"""Pins of the SpMV oracle against things other than itself."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import spmv, reorder


def dense(a):
    m = np.zeros((a.n, a.n))
    for i in range(a.n):
        for p in range(a.rowptr[i], a.rowptr[i + 1]):
            m[i, a.colidx[p]] = a.vals[p]
    return m


@pytest.mark.parametrize("n,dens,seed", [(1, 1.0, 0), (5, 0.5, 1), (17, 0.3, 2), (64, 0.1, 3),
                                         (64, 0.5, 4), (33, 0.0, 5)])
def test_brute_force_dense(n, dens, seed):
    a = synth.random_pattern(n, dens, seed, empty_rows=n // 4)
    x = synth.uniform_vector(n, seed + 100)
    ref = dense(a) @ x
    got = spmv.csr_spmv_py(a.n, a.rowptr, a.colidx, a.vals, x)
    scale = np.abs(dense(a)) @ np.abs(x)
    assert np.all(np.abs(got - ref) <= 1e-14 * scale + 0.0)
    assert np.array_equal(got, spmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x))


def test_integer_values_exact():
    a = synth.random_pattern(50, 0.3, 7, integer_values=True, empty_rows=4)
    x = np.random.default_rng(8).integers(-9, 10, size=50).astype(np.float64)
    ref = dense(a).astype(np.int64) @ x.astype(np.int64)
    got = spmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x)
    assert np.array_equal(got, ref.astype(np.float64))


def test_alpha_beta_semantics():
    a = synth.random_pattern(20, 0.3, 9)
    x = synth.uniform_vector(20, 10)
    y = synth.uniform_vector(20, 11)
    ax = dense(a) @ x
    got = spmv.csr_spmv_py(a.n, a.rowptr, a.colidx, a.vals, x, 2.5, -0.5, y)
    assert np.allclose(got, 2.5 * ax - 0.5 * y, rtol=0, atol=1e-13)
    # beta == 0: y is not read, NaN in y must not leak
    ynan = np.full(20, np.nan)
    got0 = spmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x, 1.0, 0.0, ynan)
    assert np.all(np.isfinite(got0))
    gotc = spmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x, 2.5, -0.5, y)
    assert np.array_equal(got, gotc)


def _boundary_count_2d(nx, ny):
    i = np.arange(nx * ny)
    xs, ys = i % nx, i // nx
    return (xs == 0).astype(int) + (xs == nx - 1) + (ys == 0) + (ys == ny - 1)


def test_laplacian_5pt_row_sums():
    a = synth.stencil_2d_5pt(64, 64)
    y = spmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, np.ones(a.n))
    # A*1 = 4 - #neighbours = number of missing neighbours: 0 interior, 1 edge, 2 corner
    assert np.array_equal(y, _boundary_count_2d(64, 64).astype(np.float64))
    assert sorted(np.unique(y, return_counts=True)[1].tolist()) == [4, 248, 3844]


def _missing_3d(nx, ny, nz):
    i = np.arange(nx * ny * nz)
    xs, ys, zs = i % nx, (i // nx) % ny, i // (nx * ny)
    bx = (xs == 0).astype(int) + (xs == nx - 1)
    by = (ys == 0).astype(int) + (ys == ny - 1)
    bz = (zs == 0).astype(int) + (zs == nz - 1)
    return bx, by, bz, xs, ys, zs


def test_laplacian_7pt_27pt_row_sums_and_linear():
    nx, ny, nz = 9, 7, 6
    bx, by, bz, xs, ys, zs = _missing_3d(nx, ny, nz)
    a7 = synth.stencil_3d(nx, ny, nz, 7)
    y7 = spmv.csr_spmv(a7.n, a7.rowptr, a7.colidx, a7.vals, np.ones(a7.n))
    assert np.array_equal(y7, (bx + by + bz).astype(np.float64))
    a27 = synth.stencil_3d(nx, ny, nz, 27)
    y27 = spmv.csr_spmv(a27.n, a27.rowptr, a27.colidx, a27.vals, np.ones(a27.n))
    # 26 - #neighbours; #neighbours = prod(3 - b_d) - 1 for b_d boundary sides per axis
    nb = (3 - bx) * (3 - by) * (3 - bz) - 1
    assert np.array_equal(y27, (26 - nb).astype(np.float64))
    assert set(np.unique(y27).tolist()) == {0.0, 9.0, 15.0, 19.0}
    interior = (bx + by + bz) == 0
    for lin in (xs, ys, zs, xs + 2 * ys - 3 * zs):
        for a in (a7, a27):
            y = spmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, lin.astype(np.float64))
            assert np.all(y[interior] == 0.0)


def test_csr3_loop_nest_fig1():
    # Fig. 1 pointers on a 9-row matrix: Listing 1 covers every row once and gives CSR's y.
    a = synth.random_pattern(9, 0.4, 12)
    x = synth.uniform_vector(9, 13)
    sr_ptr = np.array([0, 2, 5, 7, 9], np.int32)
    ssr_ptr = np.array([0, 2, 4], np.int32)
    y3 = spmv.csr3_spmv(ssr_ptr, sr_ptr, a.rowptr, a.colidx, a.vals, x)
    y1 = spmv.csr_spmv_py(a.n, a.rowptr, a.colidx, a.vals, x)
    assert np.array_equal(y3, y1)
    assert np.array_equal(spmv.csr3_spmv_c(ssr_ptr, sr_ptr, a.rowptr, a.colidx, a.vals, x), y1)
    # a pointer array that skips a super-row leaves rows uncovered (NaN)
    y_bad = spmv.csr3_spmv(np.array([0, 1, 4], np.int32), sr_ptr, a.rowptr, a.colidx, a.vals, x)
    assert np.isnan(y_bad).sum() == 0
    y_bad2 = spmv.csr3_spmv(np.array([0, 1, 3], np.int32), sr_ptr, a.rowptr, a.colidx, a.vals, x)
    assert np.isnan(y_bad2).sum() == 2


def test_permutation_invariance():
    # P^T (P A P^T)(P x) = A x: exactly equal, since each row keeps its entries and the
    # reorder sorts a row's columns -- with integer values any order is exact.
    a = synth.random_pattern(60, 0.15, 14, integer_values=True, symmetric=True)
    x = np.random.default_rng(15).integers(-5, 6, size=60).astype(np.float64)
    perm = reorder.rcm(a.n, a.rowptr, a.colidx)
    brp, bci, bv = reorder.permute_scipy(a.n, a.rowptr, a.colidx, a.vals, perm)
    yb = spmv.csr_spmv(a.n, brp, bci, bv, x[perm])
    y = np.empty(a.n)
    y[perm] = yb
    assert np.array_equal(y, spmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x))


def test_spmm_columns():
    a = synth.random_pattern(30, 0.2, 16, empty_rows=3)
    X = synth.uniform_block(30, 5, 17)
    Y0 = synth.uniform_block(30, 5, 18)
    Y = spmv.csr_spmm(a.n, a.rowptr, a.colidx, a.vals, X, 1.5, 0.25, Y0)
    for c in range(5):
        yc = spmv.csr_spmv_py(a.n, a.rowptr, a.colidx, a.vals, X[:, c], 1.5, 0.25, Y0[:, c])
        assert np.array_equal(Y[:, c], yc)
    assert np.allclose(Y, 1.5 * dense(a) @ X + 0.25 * Y0, atol=1e-13)


def test_rows_subset_matches_full():
    a = synth.stencil_3d(6, 6, 6, 27, "random_dd", 3)
    x = synth.uniform_vector(a.n, 2)
    y0 = synth.uniform_vector(a.n, 4)
    full = spmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x, 0.5, 2.0, y0)
    rows = np.array([0, 5, 100, a.n - 1])
    sub = spmv.csr_spmv_rows(a.rowptr, a.colidx, a.vals, x, rows, 0.5, 2.0, y0)
    assert np.array_equal(sub, full[rows])


def test_abs_scale():
    a = synth.random_pattern(20, 0.3, 19)
    x = synth.uniform_vector(20, 20)
    s = spmv.abs_row_scale(a.rowptr, a.colidx, a.vals, x)
    assert np.allclose(s, np.abs(dense(a)) @ np.abs(x), rtol=1e-15, atol=0)


@pytest.mark.parametrize("threads", [1, 2, 3, 8])
@pytest.mark.parametrize("sizes", [(32, 4), (96, 1), (7, 3)])
def test_csr3_openmp_loop_nest_matches_sequential(threads, sizes):
    """Listing 1 with its parallel loop over super-super-rows gives the sequential loop
    nest's y bit for bit, for any thread count and for CSR-2 (one super-row per
    super-super-row); every row is written exactly once."""
    from oracle import csrk as ocsrk
    a = synth.random_pattern(3001, 0.004, 17, empty_rows=40)
    x = synth.uniform_vector(a.n, 18)
    sr_ptr, ssr_ptr = ocsrk.fixed_pointers(a.n, *sizes)
    ref = spmv.csr3_spmv_c(ssr_ptr, sr_ptr, a.rowptr, a.colidx, a.vals, x)
    got, used = spmv.csr3_spmv_omp(ssr_ptr, sr_ptr, a.rowptr, a.colidx, a.vals, x, threads)
    assert np.array_equal(got, ref) and not np.isnan(got).any()
    assert 1 <= used <= threads
    assert np.array_equal(ref, spmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x))
