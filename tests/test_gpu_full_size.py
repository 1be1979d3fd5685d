"""Full-size parity: every workload the benchmark and the stated configurations name, at
its full size and with the autotuned launch shape the benchmark uses, against the oracle
on EVERY output entry (the C oracle does a whole pass over 61 M nonzeros in well under a
second) and against properties that hold at any size.

  * FEM-like SPD matrix, 160^3 jittered points (n = 4,096,000, ~61 M nonzeros);
  * the 128^3 27-point stencil with values stored FP32 and BF16 (FP64 or FP32 vectors and
    accumulation), and CG on it to 1e-10 with FP64, FP32 and BF16 inner products;
  * the 64-matrix batch (n log-uniform in [1e3, 1e6], k in {1,2,4,8,16}): one persistent
    SpMM launch and 200 CG iterations in one graph, and the batched solve to 1e-10.  The
    references start from the INPUT matrices and the oracle's own RCM permutation
    (oracle.reorder.rcm), not from anything the library exports.

Bounds: FP64 accumulation 1e-12 * s_i (s_i = sum_j |a_ij x_j|, the row's absolute scale)
against the oracle applied to the stored (rounded) values; FP32 accumulation
(m_i + 3) * 2^-24 * s_i for a row of m_i entries; CG true residuals recomputed by the
oracle's SpMV over the whole matrix."""
import numpy as np
import pytest

import synth
from oracle import precision, reorder
from oracle import spmv as ospmv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05096_gb300 import csrk  # noqa: E402

DEV = "cuda:0"


def narrowed(vals, dtype):
    if dtype == "f64":
        return vals
    if dtype == "f32":
        return precision.to_f32(vals).astype(np.float64)
    return precision.bf16_bits_to_f64(precision.to_bf16_bits(vals))


_NARROWED = {}


def narrowed_cached(a, dtype):
    """The oracle's rounding of a full-size matrix's values, computed once per dtype."""
    key = (id(a), dtype)
    if key not in _NARROWED:
        _NARROWED[key] = narrowed(a.vals, dtype)
    return _NARROWED[key]


def assert_all_rows(got, rowptr, colidx, vals, x, acc_f32=False, what=""):
    """Every entry of got against the oracle's y = A x on the same (stored) values."""
    ref = ospmv.csr_spmv(len(rowptr) - 1, rowptr, colidx, vals, x)
    s = ospmv.abs_row_scale(rowptr, colidx, vals, x)
    if acc_f32:
        m = np.diff(np.asarray(rowptr, np.int64)).astype(np.float64)
        bound = (m + 3) * 2.0 ** -24 * s
    else:
        bound = 1e-12 * s
    bad = ~(np.abs(got - ref) <= bound)
    assert not bad.any(), f"{what}: {bad.sum()} of {got.size} rows out of bound, first {np.flatnonzero(bad)[:5]}"


def spmv_device(h, x, x_f32=False, acc_f32=False):
    dt = torch.float32 if x_f32 else torch.float64
    xt = torch.tensor(x, dtype=dt, device=DEV)
    yt = torch.full_like(xt, float("nan"))
    f = (csrk.X_F32 if x_f32 else 0) | (csrk.ACC_F32 if acc_f32 else 0)
    csrk.spmv(h, 1.0, xt, 0.0, yt, f)
    torch.cuda.synchronize()
    assert csrk.device_status(h) == 0
    return yt.double().cpu().numpy()


# ------------------------------------------------------------------ FEM 160^3
@pytest.fixture(scope="module")
def fem160():
    return synth.fem_like(160, 4)


def test_fem_160cubed_autotuned(fem160):
    a = fem160
    assert a.n == 160 ** 3 and 55e6 < a.nnz < 67e6
    rl = np.diff(a.rowptr)
    assert 12 <= rl.min() - 1 and rl.var() <= 10          # 12-18 neighbours (+ diagonal), variance <= 10
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, "f64")
    csrk.reorder(h)
    csrk.set_sizes(h, 0, 0)                                # the benchmark's autotuned shape
    x = synth.uniform_vector(a.n, 2)
    got = spmv_device(h, x)
    assert_all_rows(got, a.rowptr, a.colidx, a.vals, x, what=f"FEM {csrk.tuned_config(h)}")
    # every row: A 1 is the row sum (in any summation order, within 1e-12 of the row's
    # absolute sum)
    ones = spmv_device(h, np.ones(a.n))
    rs = np.add.reduceat(a.vals, a.rowptr[:-1])
    ra = np.add.reduceat(np.abs(a.vals), a.rowptr[:-1])
    assert np.all(np.abs(ones - rs) <= 1e-12 * ra)
    csrk.destroy(h)


# ------------------------------------------------------------------ 27-point precision
@pytest.fixture(scope="module")
def st27():
    n = 128 ** 3
    return synth.stencil_3d(128, 128, 128, 27, "random_dd", 3, labels=synth.vectors.permutation(n, 3))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("mode", ["x64acc64", "x32acc32"])
def test_27pt_128cubed_narrow_values(st27, dtype, mode):
    a = st27
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, dtype)
    csrk.reorder(h)
    csrk.set_sizes(h, 0, 0)
    x = synth.uniform_vector(a.n, 2)
    x_f32 = acc_f32 = mode == "x32acc32"
    got = spmv_device(h, x, x_f32, acc_f32)
    xr = x.astype(np.float32).astype(np.float64) if x_f32 else x
    v = narrowed_cached(a, dtype)
    assert_all_rows(got, a.rowptr, a.colidx, v, xr, acc_f32, what=f"{dtype} {mode} {csrk.tuned_config(h)}")
    csrk.destroy(h)


def test_27pt_128cubed_cg_fp64_and_mixed(st27):
    a = st27
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, "f64")
    csrk.reorder(h)
    csrk.set_sizes(h, 0, 0)
    b = synth.uniform_vector(a.n, 5)
    bt = torch.tensor(b, device=DEV)
    its = {}
    for inner, restart in (("f64", 0), ("f32", 0), ("bf16", 1)):
        xt = torch.zeros_like(bt)
        rc, it, rel = csrk.cg(h, bt, xt, 1e-10, 5000, inner, 20, restart)
        assert rc == 0 and rel <= 1e-10, (inner, rc, it, rel)
        x = xt.cpu().numpy()
        true = np.linalg.norm(b - ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x)) / np.linalg.norm(b)
        assert true <= 1.05e-10, (inner, true)
        its[inner] = it
    assert its["f32"] <= 1.3 * its["f64"] + 20 and its["bf16"] <= 2.0 * its["f64"] + 40, its
    csrk.destroy(h)


# ------------------------------------------------------------------ the 64-matrix batch
@pytest.fixture(scope="module")
def batch64():
    """The batch's input matrices, the oracle's RCM permutation of each (the library's
    reordering is held to it bit for bit elsewhere), and the library's batch over them."""
    specs = synth.batch_specs()
    hs, mats, perms, ks = [], [], [], []
    for sp in specs:
        a = synth.batch_matrix(sp)
        h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, sp["dtype"])
        csrk.reorder(h, "rcm", want_perm=False)
        csrk.set_sizes(h, 0, 0)
        mats.append((a, sp["dtype"]))
        perms.append(reorder.rcm(a.n, a.rowptr, a.colidx))
        hs.append(h)
        ks.append(sp["k"])
    b = csrk.batch_create(hs, ks)
    yield hs, mats, perms, ks, b
    csrk.batch_destroy(b)
    for h in hs:
        csrk.destroy(h)


def _to_reordered(x_in, perm):
    """Block of vectors in the input numbering -> the reordered numbering (row i of the
    result is row perm[i] of the input)."""
    return np.ascontiguousarray(x_in[perm])


def test_batch64_spmm_every_row(batch64):
    """Y = A X for each matrix, in the reordered numbering the batch works in: Y[i] must
    equal (A x_in)[perm[i]] with X[i] = x_in[perm[i]], A the input matrix."""
    hs, mats, perms, ks, b = batch64
    assert len(hs) == 64 and 140e6 < sum(a.nnz for a, _ in mats) < 160e6
    Xin = [synth.uniform_block(a.n, k, 500 + i) for i, ((a, _), k) in enumerate(zip(mats, ks))]
    Xs = [torch.tensor(_to_reordered(X, p), device=DEV) for X, p in zip(Xin, perms)]
    Ys = [torch.full_like(x, float("nan")) for x in Xs]
    csrk.batch_spmm(b, 1.0, Xs, 0.0, Ys)
    torch.cuda.synchronize()
    assert csrk.batch_device_status(b) == 0
    for i, ((a, dtype), k) in enumerate(zip(mats, ks)):
        Y = Ys[i].cpu().numpy()
        y_in = np.empty_like(Y)
        y_in[perms[i]] = Y
        vv = narrowed(a.vals, dtype)
        for c in range(k):
            assert_all_rows(np.ascontiguousarray(y_in[:, c]), a.rowptr, a.colidx, vv,
                            np.ascontiguousarray(Xin[i][:, c]), what=f"matrix {i} column {c}")


def test_batch64_cg_200_iterations_and_solve(batch64):
    """Solutions checked by their true residuals ||b - A x|| / ||b|| on the input matrices
    (x and b brought back to the input numbering through the oracle's permutation)."""
    hs, mats, perms, ks, b = batch64
    Bin = [synth.uniform_block(a.n, k, 700 + i) for i, ((a, _), k) in enumerate(zip(mats, ks))]
    Bs = [torch.tensor(_to_reordered(B, p), device=DEV) for B, p in zip(Bin, perms)]

    def true_residuals(Xs, operator_values):
        out = []
        for i, ((a, dtype), k) in enumerate(zip(mats, ks)):
            X = Xs[i].cpu().numpy()
            x_in = np.empty_like(X)
            x_in[perms[i]] = X
            vv = operator_values(a, dtype)
            for c in range(k):
                r = Bin[i][:, c] - ospmv.csr_spmv(a.n, a.rowptr, a.colidx, vv, np.ascontiguousarray(x_in[:, c]))
                out.append(np.linalg.norm(r) / np.linalg.norm(Bin[i][:, c]))
        return np.array(out)

    # 200 iterations in one graph, on the stored operator: every system reaches 1e-10
    Xs = [torch.zeros_like(x) for x in Bs]
    rel, its = csrk.batch_cg(b, Bs, Xs, 200, 1e-10)
    assert rel.size == sum(ks) and np.all(rel <= 1.05e-10), (np.count_nonzero(rel > 1.05e-10), rel.max())
    true = true_residuals(Xs, lambda a, dtype: narrowed(a.vals, dtype))
    assert np.all(true <= 1.05e-10), (np.argmax(true), true.max())
    assert np.all(np.abs(true - rel) <= 1e-12 + 1e-3 * true)
    # the solve to 1e-10 on the FP64 operator, FP32 inner products
    Xs = [torch.zeros_like(x) for x in Bs]
    rc, rel, its, cycles = csrk.batch_cg_solve(b, Bs, Xs, rtol=1e-10, maxit=2000, inner="f32")
    assert rc == 0 and np.all(rel <= 1e-10)
    true = true_residuals(Xs, lambda a, dtype: a.vals)
    assert np.all(true <= 1.05e-10), (np.argmax(true), true.max())
    assert csrk.batch_device_status(b) == 0
