"""Oracle SpMV / SpMM (TEST INFRASTRUCTURE).

What the method computes (Sec. 1, problem statement "Ax = y"; Listing 1's innermost loop):
for every row i, y_i is the sum over the row's stored nonzeros of a_ij * x_j.  The CSR-k
structure (Sec. 2.2) only groups rows; it never changes a row's arithmetic.  The library's
interface adds the BLAS scaling y = alpha*A*x + beta*y; beta == 0 means y is not read.

Arithmetic: FP64, the row's entries added left to right in stored order, each product
rounded before the add (Python floats; the C twin is built without FMA).

Pins (tests/test_oracle_spmv.py): dense brute force on random patterns up to n = 64,
including empty rows; exact results for integer-valued inputs; the closed-form row sums of
5-, 7- and 27-point Laplacians applied to the ones vector and to linear vectors; the
CSR-3 loop nest of Listing 1 on the Fig. 1 pointer example; permutation invariance
P^T (P A P^T)(P x) = A x; the C twin agreeing bit for bit.
"""
from __future__ import annotations

import numpy as np

from . import native


def csr_spmv_py(n, rowptr, colidx, vals, x, alpha=1.0, beta=0.0, y=None):
    """Row-by-row CSR SpMV in pure Python loops (small inputs only)."""
    out = np.empty(n, dtype=np.float64)
    for i in range(n):
        s = 0.0
        for p in range(int(rowptr[i]), int(rowptr[i + 1])):
            s = s + float(vals[p]) * float(x[int(colidx[p])])
        if beta == 0.0:
            out[i] = alpha * s
        else:
            out[i] = alpha * s + beta * float(y[i])
    return out


def csr_spmv(n, rowptr, colidx, vals, x, alpha=1.0, beta=0.0, y=None):
    """Same arithmetic as csr_spmv_py, in the C twin (any size)."""
    out = np.array(y, dtype=np.float64, copy=True) if (beta != 0.0) else np.empty(n)
    native.lib().oracle_csr_spmv(int(n), np.ascontiguousarray(rowptr, np.int32),
                                 np.ascontiguousarray(colidx, np.int32),
                                 np.ascontiguousarray(vals, np.float64),
                                 np.ascontiguousarray(x, np.float64), float(alpha),
                                 float(beta), out)
    return out


def csr_spmv_rows(rowptr, colidx, vals, x, rows, alpha=1.0, beta=0.0, y=None):
    """Oracle values of the selected rows only (full-size sampled checks)."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(rows.size, dtype=np.float64)
    yarr = None
    if beta != 0.0:
        yarr = np.ascontiguousarray(y, dtype=np.float64)
    native.lib().oracle_csr_spmv_rows(np.ascontiguousarray(rowptr, np.int32),
                                      np.ascontiguousarray(colidx, np.int32),
                                      np.ascontiguousarray(vals, np.float64),
                                      np.ascontiguousarray(x, np.float64), float(alpha),
                                      float(beta),
                                      None if yarr is None else yarr.ctypes.data,
                                      rows, rows.size, out)
    return out


def csr3_spmv(ssr_ptr, sr_ptr, rowptr, colidx, vals, x):
    """Listing 1 (CSR-3 kernel): super-super-rows -> super-rows -> rows -> nonzeros.

    Returns y with y[k] = sum of the row's products; rows not covered by any super-row
    stay NaN, so a pointer array that misses rows shows up in the comparison.
    """
    n = len(rowptr) - 1
    y = np.full(n, np.nan)
    num_ssr = len(ssr_ptr) - 1
    for i in range(num_ssr):
        for j in range(int(ssr_ptr[i]), int(ssr_ptr[i + 1])):
            for k in range(int(sr_ptr[j]), int(sr_ptr[j + 1])):
                temp = 0.0
                for l in range(int(rowptr[k]), int(rowptr[k + 1])):
                    temp = temp + float(vals[l]) * float(x[int(colidx[l])])
                y[k] = temp
    return y


def csr3_spmv_c(ssr_ptr, sr_ptr, rowptr, colidx, vals, x):
    """Listing 1 in the C twin."""
    n = len(rowptr) - 1
    y = np.full(n, np.nan)
    native.lib().oracle_csr3_spmv(int(len(ssr_ptr) - 1), np.ascontiguousarray(ssr_ptr, np.int32),
                                  np.ascontiguousarray(sr_ptr, np.int32),
                                  np.ascontiguousarray(rowptr, np.int32),
                                  np.ascontiguousarray(colidx, np.int32),
                                  np.ascontiguousarray(vals, np.float64),
                                  np.ascontiguousarray(x, np.float64), y)
    return y


def csr3_spmv_omp(ssr_ptr, sr_ptr, rowptr, colidx, vals, x, threads=0, out=None):
    """Listing 1 with its OpenMP parallel loop over super-super-rows (static schedule), in
    the C twin.  Returns (y, threads used); y is bit-identical to csr3_spmv_c."""
    n = len(rowptr) - 1
    y = np.full(n, np.nan) if out is None else out
    used = native.lib().oracle_csr3_spmv_omp(int(len(ssr_ptr) - 1), np.ascontiguousarray(ssr_ptr, np.int32),
                                             np.ascontiguousarray(sr_ptr, np.int32),
                                             np.ascontiguousarray(rowptr, np.int32),
                                             np.ascontiguousarray(colidx, np.int32),
                                             np.ascontiguousarray(vals, np.float64),
                                             np.ascontiguousarray(x, np.float64), y, int(threads))
    return y, int(used)


def csr_spmm(n, rowptr, colidx, vals, X, alpha=1.0, beta=0.0, Y=None):
    """Y = alpha*A*X + beta*Y for k right-hand sides (X, Y row-major n x k): each column
    is exactly csr_spmv of that column."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    k = X.shape[1]
    out = np.array(Y, dtype=np.float64, copy=True) if beta != 0.0 else np.empty((n, k))
    native.lib().oracle_csr_spmm(int(n), np.ascontiguousarray(rowptr, np.int32),
                                 np.ascontiguousarray(colidx, np.int32),
                                 np.ascontiguousarray(vals, np.float64), int(k),
                                 X.reshape(-1), int(k), float(alpha), float(beta),
                                 out.reshape(-1), int(k))
    return out


def abs_row_scale(rowptr, colidx, vals, x, alpha=1.0, beta=0.0, y=None, rows=None):
    """s_i = |alpha| * sum_j |a_ij x_j| + |beta| |y_i|: the per-entry normaliser of the
    error bounds.  Computed with the same oracle loop on |A| and |x|."""
    if rows is None:
        n = len(rowptr) - 1
        s = csr_spmv(n, rowptr, colidx, np.abs(vals), np.abs(x), abs(alpha), 0.0)
        if beta != 0.0:
            s = s + abs(beta) * np.abs(y)
        return s
    s = csr_spmv_rows(rowptr, colidx, np.abs(vals), np.abs(x), rows, abs(alpha), 0.0)
    if beta != 0.0:
        s = s + abs(beta) * np.abs(np.asarray(y)[np.asarray(rows)])
    return s
