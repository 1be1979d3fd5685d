"""Oracle conjugate gradients, FP64 and mixed precision (TEST INFRASTRUCTURE).

The paper names CG on PDE matrices as the consumer of its SpMV (Sec. 1, Sec. 5.3, Sec. 8, Sec. 9);
the library adds an FP64 CG and a mixed-precision CG on top of its kernels.  The reading
used by both this oracle and the library:

FP64 CG (Hestenes-Stiefel): x0 = 0, r0 = b, p0 = r0;
    q = A p;  alpha = (r.r) / (p.q);  x += alpha p;  r -= alpha q;
    beta = (r'.r') / (r.r);  p = r' + beta p.
Stops when the recursively updated ||r|| / ||b|| <= rtol; the true residual
||b - A x|| / ||b|| is reported beside it.

Mixed-precision CG: the same recurrences with every vector, dot product, alpha and beta in
FP64, but q = A_lo p uses A's values rounded to FP32 or BF16 (and p rounded to FP32).
Every ``replace_every`` iterations, or earlier once the recursive residual has dropped
below rtol/2, the residual is recomputed in FP64, r = b - A x with the FP64 values.  With
``restart`` the search direction is then reset, p = r (defect correction: each cycle is a
short CG on the correction equation).  Without it p is kept (reliable-update CG) unless
the recomputed residual norm exceeds twice the recursive one, or the recursive residual
norm grew tenfold within the cycle: then the kept direction no longer matches the
residual it is meant to reduce, and the cycle ends with a restart too.  The
solve stops when a recomputed FP64 residual satisfies rtol.  Breakdown (p.q <= 0 or
r.r == 0) stops the iteration.

Pins (tests/test_oracle_cg.py): small SPD systems against numpy.linalg.solve; FP64 CG on
the 1-D Laplacian reaches the solution within n iterations (finite termination in exact
arithmetic); the mixed solve's final residual recomputed independently.
"""
from __future__ import annotations

import numpy as np

from . import precision
from .spmv import csr_spmv


def _norm(v):
    return float(np.sqrt(np.dot(v, v)))


def cg_fp64(n, rowptr, colidx, vals, b, rtol=1e-10, maxit=10000):
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(n)
    r = b.copy()
    p = r.copy()
    rr = float(np.dot(r, r))
    bnorm = _norm(b)
    it = 0
    if bnorm == 0.0:
        return x, 0, 0.0
    while it < maxit and np.sqrt(rr) / bnorm > rtol:
        q = csr_spmv(n, rowptr, colidx, vals, p)
        pq = float(np.dot(p, q))
        if pq <= 0.0 or rr == 0.0:
            break
        alpha = rr / pq
        x += alpha * p
        r -= alpha * q
        rr_new = float(np.dot(r, r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    true_res = _norm(b - csr_spmv(n, rowptr, colidx, vals, x)) / bnorm
    return x, it, true_res


def lowered_values(vals, lo):
    """A's values as the low-precision SpMV sees them (exactly widened back to FP64)."""
    if lo == "f32":
        return precision.to_f32(vals).astype(np.float64)
    if lo == "bf16":
        return precision.bf16_bits_to_f64(precision.to_bf16_bits(vals))
    raise ValueError(lo)


def cg_mixed(n, rowptr, colidx, vals, b, lo="f32", rtol=1e-10, maxit=10000,
             replace_every=20, restart=True, vals_lo=None):
    b = np.asarray(b, dtype=np.float64)
    a_lo = lowered_values(vals, lo) if vals_lo is None else vals_lo
    bnorm = _norm(b)
    x = np.zeros(n)
    if bnorm == 0.0:
        return x, 0, 0.0
    r = b.copy()
    p = r.copy()
    rr = float(np.dot(r, r))
    it = 0
    true_res = 1.0
    while it < maxit:
        rr_start = rr
        diverged = False
        for _ in range(replace_every):
            p_lo = p.astype(np.float32).astype(np.float64)
            q = csr_spmv(n, rowptr, colidx, a_lo, p_lo)
            pq = float(np.dot(p, q))
            if pq <= 0.0 or rr == 0.0:
                break
            alpha = rr / pq
            x += alpha * p
            r -= alpha * q
            rr_new = float(np.dot(r, r))
            p = r + (rr_new / rr) * p
            rr = rr_new
            it += 1
            if rr > 100.0 * rr_start:
                diverged = True
                break
            if it >= maxit or np.sqrt(rr) <= 0.5 * rtol * bnorm:
                break
        rr_rec = rr
        r = b - csr_spmv(n, rowptr, colidx, vals, x)
        rr = float(np.dot(r, r))
        true_res = np.sqrt(rr) / bnorm
        if true_res <= rtol or rr == 0.0:
            break
        if restart or diverged or rr > 4.0 * rr_rec:
            p = r.copy()
    return x, it, true_res
