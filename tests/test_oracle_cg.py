"""Pins of the CG oracle."""
import numpy as np
import pytest

import synth
from oracle import cg, spmv


def test_small_spd_against_solve():
    a = synth.stencil_3d(6, 5, 4, 27, "random_dd", 3)
    b = synth.uniform_vector(a.n, 5)
    A = np.zeros((a.n, a.n))
    for i in range(a.n):
        A[i, a.colidx[a.rowptr[i]:a.rowptr[i + 1]]] = a.vals[a.rowptr[i]:a.rowptr[i + 1]]
    xs = np.linalg.solve(A, b)
    x, it, res = cg.cg_fp64(a.n, a.rowptr, a.colidx, a.vals, b, 1e-12)
    assert res <= 1e-11 and np.allclose(x, xs, rtol=0, atol=1e-9 * np.abs(xs).max())
    for lo in ("f32", "bf16"):
        for restart in (True, False):
            x2, it2, res2 = cg.cg_mixed(a.n, a.rowptr, a.colidx, a.vals, b, lo, 1e-10, 2000, 20, restart)
            true = np.linalg.norm(b - A @ x2) / np.linalg.norm(b)
            assert res2 <= 1e-10 and true <= 1.01e-10


def test_1d_laplacian_finite_termination():
    n = 50
    rows, cols, vals = [], [], []
    for i in range(n):
        for j, v in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                rows.append(i); cols.append(j); vals.append(v)
    a = synth.matrices._from_coo(n, np.array(rows), np.array(cols), np.array(vals))
    b = synth.uniform_vector(n, 1)
    x, it, res = cg.cg_fp64(n, a.rowptr, a.colidx, a.vals, b, 1e-10)
    assert it <= n + 5 and res <= 1e-9


def test_zero_rhs():
    a = synth.stencil_2d_5pt(4, 4)
    x, it, res = cg.cg_fp64(a.n, a.rowptr, a.colidx, a.vals, np.zeros(a.n))
    assert it == 0 and np.all(x == 0)


def test_lowered_values():
    v = np.array([1 + 2**-8 + 2**-40, 0.1])
    assert cg.lowered_values(v, "bf16")[0] == 1 + 2**-7
    assert cg.lowered_values(v, "f32")[1] == float(np.float32(0.1))
