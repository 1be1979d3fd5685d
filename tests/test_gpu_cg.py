"""GPU conjugate gradients (FP64 and mixed precision, graph-captured) against the oracle.

Pass criteria: the library's own true residual ||b - A x|| / ||b|| <= rtol, recomputed
independently here with the oracle SpMV on the returned x; the solution agrees with
numpy.linalg.solve within cond(A) * rtol; iteration counts stay close to the oracle CG's
(the GPU sums in a different order, so counts may differ by a few)."""
import numpy as np
import pytest

import synth
from oracle import cg as ocg
from oracle import spmv as ospmv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05096_gb300 import csrk  # noqa: E402

DEV = "cuda:0"


def setup(a, sizes=(32, 4)):
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder(h)
    csrk.set_sizes(h, *sizes)
    return h


def true_relres(a, x, b):
    r = b - ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("inner,restart", [("f64", 0), ("f32", 0), ("f32", 1), ("bf16", 1), ("bf16", 0)])
def test_cg_converges_and_matches_oracle(inner, restart):
    a = synth.stencil_3d(24, 22, 20, 27, "random_dd", 3, labels=synth.vectors.permutation(24 * 22 * 20, 3))
    b = synth.uniform_vector(a.n, 5)
    h = setup(a)
    bt = torch.tensor(b, device=DEV)
    xt = torch.zeros_like(bt)
    rc, iters, rel = csrk.cg(h, bt, xt, 1e-10, 3000, inner, 20, restart)
    x = xt.cpu().numpy()
    assert rc == 0, (rc, iters, rel)
    assert rel <= 1e-10
    assert true_relres(a, x, b) <= 1.05e-10
    if inner == "f64":
        _, it_ref, _ = ocg.cg_fp64(a.n, a.rowptr, a.colidx, a.vals, b, 1e-10)
        assert abs(iters - it_ref) <= 3
    else:
        _, it_ref, _ = ocg.cg_mixed(a.n, a.rowptr, a.colidx, a.vals, b, inner, 1e-10, 3000, 20, bool(restart))
        assert iters <= 1.3 * it_ref + 20
    csrk.destroy(h)


def test_cg_solution_vs_dense_solve_and_graph_reuse():
    a = synth.stencil_3d(9, 8, 7, 27, "random_dd", 4)
    A = np.zeros((a.n, a.n))
    for i in range(a.n):
        A[i, a.colidx[a.rowptr[i]:a.rowptr[i + 1]]] = a.vals[a.rowptr[i]:a.rowptr[i + 1]]
    h = setup(a, (16, 2))
    for seed in (6, 7):                       # second solve replays the captured graph
        b = synth.uniform_vector(a.n, seed)
        xs = np.linalg.solve(A, b)
        bt = torch.tensor(b, device=DEV)
        xt = torch.zeros_like(bt)
        rc, iters, rel = csrk.cg(h, bt, xt, 1e-12, 1000, "f64")
        assert rc == 0 and rel <= 1e-12
        assert np.allclose(xt.cpu().numpy(), xs, rtol=0, atol=1e-9 * np.abs(xs).max())
    csrk.destroy(h)


def test_cg_1d_laplacian_finite_termination():
    n = 300
    rows, cols, vals = [], [], []
    for i in range(n):
        for j, v in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                rows.append(i); cols.append(j); vals.append(v)
    a = synth.matrices._from_coo(n, np.array(rows), np.array(cols), np.array(vals))
    h = setup(a, (32, 2))
    b = synth.uniform_vector(n, 1)
    bt = torch.tensor(b, device=DEV)
    xt = torch.zeros_like(bt)
    rc, iters, rel = csrk.cg(h, bt, xt, 1e-10, 2 * n, "f64")
    assert rc == 0 and iters <= n + 10
    csrk.destroy(h)


def test_cg_permuted_vectors_and_iteration_limit():
    a = synth.stencil_3d(12, 12, 12, 7, "random_dd", 8, labels=synth.vectors.permutation(1728, 8))
    b = synth.uniform_vector(a.n, 9)
    h = setup(a)
    perm = csrk.export(h)["perm"]
    bt = torch.tensor(b[perm], device=DEV)
    xt = torch.zeros_like(bt)
    rc, iters, rel = csrk.cg(h, bt, xt, 1e-10, 1000, "f32", 20, 0, flags=csrk.VEC_PERMUTED)
    assert rc == 0
    x = np.empty(a.n)
    x[perm] = xt.cpu().numpy()
    assert true_relres(a, x, b) <= 1.05e-10
    rc, iters, rel = csrk.cg(h, torch.tensor(b, device=DEV), torch.zeros_like(bt), 1e-14, 5, "f64")
    assert rc == 8 and iters == 5 and rel > 1e-14      # CSRK_ERR_NOT_CONVERGED at maxit
    csrk.destroy(h)


def test_cg_zero_rhs():
    a = synth.stencil_3d(6, 6, 6, 7, "random_dd", 2)
    h = setup(a, (8, 2))
    bt = torch.zeros(a.n, dtype=torch.float64, device=DEV)
    xt = torch.full_like(bt, 7.0)
    rc, iters, rel = csrk.cg(h, bt, xt, 1e-10, 100, "f64")
    assert rc == 0 and iters == 0 and torch.all(xt == 0)
    csrk.destroy(h)


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_cg_kernel_choice_and_determinism(inner):
    """The solve's SpMV on the staged kernel (0), the staged kernel with 16-bit column
    codes (4) and the direct kernel (1): each converges to the oracle-checked residual,
    iteration counts within 2 of each other, and each is deterministic (two solves give
    bit-identical x)."""
    a = synth.stencil_3d(22, 20, 18, 27, "random_dd", 11, labels=synth.vectors.permutation(22 * 20 * 18, 11))
    b = synth.uniform_vector(a.n, 12)
    h = setup(a)
    bt = torch.tensor(b, device=DEV)
    its, xs = {}, {}
    for kernel in (0, 4, 1):
        csrk.set_config(h, kernel=kernel, lanes=1, unroll=8, warps=16, ctas=2 if kernel != 1 else -1)
        runs = []
        for _ in range(2):
            xt = torch.zeros_like(bt)
            rc, iters, rel = csrk.cg(h, bt, xt, 1e-10, 3000, inner, 20, 0)
            assert rc == 0 and rel <= 1e-10, (kernel, rc, iters, rel)
            runs.append((iters, xt.cpu().numpy()))
        assert runs[0][0] == runs[1][0] and np.array_equal(runs[0][1], runs[1][1])
        assert true_relres(a, runs[0][1], b) <= 1.05e-10
        its[kernel], xs[kernel] = runs[0]
    assert abs(its[0] - its[1]) <= 2 and abs(its[4] - its[1]) <= 2, its
    assert csrk.device_status(h) == 0
    csrk.destroy(h)


@pytest.mark.parametrize("kernel", [0, 1])
def test_cg_breakdown_on_indefinite_matrix(kernel):
    """A negative definite matrix (the negated 1-D Laplacian) gives p.q < 0 at the first
    iteration: the solve stops with CSRK_ERR_NOT_CONVERGED, no iteration done and the
    breakdown named, on the staged (0) and the direct (1) kernel."""
    n = 300
    rows, cols, vals = [], [], []
    for i in range(n):
        for j, v in ((i - 1, 1.0), (i, -2.0), (i + 1, 1.0)):
            if 0 <= j < n:
                rows.append(i); cols.append(j); vals.append(v)
    a = synth.matrices._from_coo(n, np.array(rows), np.array(cols), np.array(vals))
    h = setup(a, (32, 2))
    csrk.set_config(h, kernel=kernel, lanes=1, unroll=8, warps=16, ctas=2 if kernel == 0 else -1)
    bt = torch.tensor(synth.uniform_vector(n, 3), device=DEV)
    rc, iters, rel = csrk.cg(h, bt, torch.zeros_like(bt), 1e-10, 100, "f64")
    assert rc == 8 and iters == 0, (rc, iters, rel)
    assert "breakdown" in csrk.lib().csrk_last_error().decode()
    csrk.destroy(h)
