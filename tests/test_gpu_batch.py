"""Batched persistent SpMM and batched CG over matrices of uneven size, against the oracle."""
import numpy as np
import pytest

import synth
from oracle import cg as ocg
from oracle import precision
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


def make_batch(specs):
    """specs: list of (CSR, dtype, k, (sr, ssr)); returns handles, exported reordered CSRs."""
    hs, forms = [], []
    for a, dtype, k, sizes in specs:
        h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, dtype)
        csrk.reorder(h)
        csrk.set_sizes(h, *sizes)
        e = csrk.export(h)
        forms.append((e["rowptr"], e["colidx"], narrowed(e["vals"], dtype)))
        hs.append(h)
    return hs, forms


SPECS = [
    (synth.stencil_3d(17, 13, 11, 27, "random_dd", 1), "f64", 1, (32, 4)),
    (synth.stencil_3d(23, 19, 7, 7, "random_dd", 2), "f32", 2, (16, 8)),
    (synth.fem_like(9, 3), "f64", 3, (32, 2)),
    (synth.stencil_3d(5, 5, 5, 27, "random_dd", 4), "bf16", 4, (8, 3)),
    (synth.random_pattern(333, 0.02, 5, symmetric=True, empty_rows=11), "f64", 8, (32, 8)),
    (synth.stencil_3d(31, 29, 3, 7, "random_dd", 6), "f64", 16, (64, 2)),
    (synth.stencil_2d_5pt(20, 9), "f32", 33, (32, 1)),
]


# item budgets: the default (16 KB), one super-row per item (many small stages), and a
# budget so large that two stages cannot fit and the direct-load kernel runs
ITEM_BUDGETS = {"default": None, "one_sr_per_item": "1", "direct": str(1 << 30)}


@pytest.mark.parametrize("budget", list(ITEM_BUDGETS))
def test_batch_spmm_matches_oracle_and_replays(budget, monkeypatch):
    if ITEM_BUDGETS[budget] is None:
        monkeypatch.delenv("CSRK_BATCH_ITEM_BYTES", raising=False)
    else:
        monkeypatch.setenv("CSRK_BATCH_ITEM_BYTES", ITEM_BUDGETS[budget])
    hs, forms = make_batch(SPECS)
    ks = [k for _, _, k, _ in SPECS]
    b = csrk.batch_create(hs, ks)
    info = csrk.batch_info(b)
    assert info["nmat"] == len(SPECS) and info["nsys"] == sum(ks)
    plan = csrk.batch_plan(b)
    if budget == "direct":
        assert plan["stages"] == 0 and plan["items"] == 0
    else:
        assert 2 <= plan["stages"] <= 16 and plan["items"] >= len(SPECS)
    if budget == "one_sr_per_item":
        nsr = sum(csrk.info(h)["nsr"] for h in hs)
        assert plan["items"] == nsr
    Xs, Ys, Y0s = [], [], []
    for i, (a, _, k, _) in enumerate(SPECS):
        X = synth.uniform_block(a.n, k, 100 + i)
        Y0 = synth.uniform_block(a.n, k, 200 + i)
        Xs.append(torch.tensor(X, device=DEV))
        Ys.append(torch.tensor(Y0, device=DEV))
        Y0s.append(Y0)
    for rep in range(3):                        # the tile counter resets itself between launches
        for i in range(len(SPECS)):
            Ys[i].copy_(torch.tensor(Y0s[i], device=DEV))
        csrk.batch_spmm(b, 1.5, Xs, -0.5, Ys)
        torch.cuda.synchronize()
        for i, ((a, _, k, _), (rp, ci, v)) in enumerate(zip(SPECS, forms)):
            X = Xs[i].cpu().numpy()
            ref = ospmv.csr_spmm(a.n, rp, ci, v, X, 1.5, -0.5, Y0s[i])
            got = Ys[i].cpu().numpy()
            for c in range(k):
                s = ospmv.abs_row_scale(rp, ci, v, X[:, c], 1.5, -0.5, Y0s[i][:, c])
                assert np.all(np.abs(got[:, c] - ref[:, c]) <= 1e-12 * s), (i, c, rep)
    # new output buffers: the bound table is rebuilt
    Zs = [torch.zeros_like(y) for y in Ys]
    csrk.batch_spmm(b, 1.0, Xs, 0.0, Zs)
    torch.cuda.synchronize()
    (rp, ci, v), (a, _, k, _) = forms[0], SPECS[0]
    ref = ospmv.csr_spmm(a.n, rp, ci, v, Xs[0].cpu().numpy())
    assert np.allclose(Zs[0].cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert csrk.batch_device_status(b) == 0
    csrk.batch_destroy(b)
    for h in hs:
        csrk.destroy(h)


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("aligned", [True, False])
def test_batch_spmm_vector_and_scalar_paths(fp32, aligned):
    """Power-of-two k on 16-byte aligned blocks take the vector-load row routines; views one
    element off a 16-byte boundary take the scalar ones.  FP32 mode: FP32 vectors and
    accumulation on the values rounded to FP32 (BF16 stays BF16)."""
    specs = [s for s in SPECS if s[2] != 33] + [(synth.stencil_3d(9, 8, 7, 27, "random_dd", 12), "f64", 32, (32, 2))]
    hs, forms = make_batch(specs)
    b = csrk.batch_create(hs, [k for _, _, k, _ in specs])
    dt = torch.float32 if fp32 else torch.float64
    flags = csrk.VEC_PERMUTED | (csrk.X_F32 | csrk.ACC_F32 if fp32 else 0)
    Xs, Ys, bufs = [], [], []
    for i, (a, _, k, _) in enumerate(specs):
        X = synth.uniform_block(a.n, k, 800 + i)
        if fp32:
            X = precision.to_f32(X).astype(np.float64)          # exactly representable in FP32
        off = 0 if aligned else 1
        bx = torch.zeros(a.n * k + 4, dtype=dt, device=DEV)
        by = torch.full((a.n * k + 4,), np.nan, dtype=dt, device=DEV)
        bx[off:off + a.n * k] = torch.tensor(X.ravel(), dtype=dt, device=DEV)
        Xs.append(bx[off:off + a.n * k].view(a.n, k))
        Ys.append(by[off:off + a.n * k].view(a.n, k))
        bufs.append((bx, by))
    csrk.batch_spmm(b, 1.0, Xs, 0.0, Ys, flags=flags)
    torch.cuda.synchronize()
    for i, ((a, dtype, k, _), (rp, ci, v)) in enumerate(zip(specs, forms)):
        X = Xs[i].double().cpu().numpy()
        got = Ys[i].double().cpu().numpy()
        vv = v if not fp32 or dtype == "bf16" else precision.to_f32(v).astype(np.float64)
        ref = ospmv.csr_spmm(a.n, rp, ci, vv, X)
        m = int(np.max(np.diff(rp)))
        tol = (m + 2) * 2.0 ** -24 if fp32 else 1e-12
        for c in range(k):
            s_ = ospmv.abs_row_scale(rp, ci, vv, X[:, c])
            assert np.all(np.abs(got[:, c] - ref[:, c]) <= tol * s_), (i, c)
    assert csrk.batch_device_status(b) == 0
    csrk.batch_destroy(b)
    for h in hs:
        csrk.destroy(h)


def test_batch_spmm_many_items_per_block():
    """Enough items that every block's stage ring wraps many times (sampled rows)."""
    specs = [(synth.stencil_3d(64, 64, 64, 27, "random_dd", 21), "f64", 4, (32, 4)),
             (synth.stencil_3d(80, 80, 80, 7, "random_dd", 22), "f32", 1, (32, 8)),
             (synth.fem_like(40, 23), "f64", 8, (32, 2))]
    hs, forms = make_batch(specs)
    b = csrk.batch_create(hs, [k for _, _, k, _ in specs])
    plan = csrk.batch_plan(b)
    assert plan["stages"] >= 2 and plan["items"] > plan["stages"] * 304   # rings wrap
    Xs = [torch.tensor(synth.uniform_block(a.n, k, 400 + i), device=DEV) for i, (a, _, k, _) in enumerate(specs)]
    Ys = [torch.full_like(x, np.nan) for x in Xs]
    for _ in range(2):
        csrk.batch_spmm(b, 1.0, Xs, 0.0, Ys)
    torch.cuda.synchronize()
    assert csrk.batch_device_status(b) == 0
    rng = np.random.default_rng(5)
    for i, ((a, _, k, _), (rp, ci, v)) in enumerate(zip(specs, forms)):
        rows = np.unique(np.concatenate([rng.integers(0, a.n, 3000), [0, a.n - 1]]))
        X, got = Xs[i].cpu().numpy(), Ys[i].cpu().numpy()
        for c in range(k):
            ref = ospmv.csr_spmv_rows(rp, ci, v, X[:, c], rows)
            s = ospmv.abs_row_scale(rp, ci, v, X[:, c], rows=rows)
            assert np.all(np.abs(got[rows, c] - ref) <= 1e-12 * s), (i, c)
        assert not np.isnan(got).any()
    csrk.batch_destroy(b)
    for h in hs:
        csrk.destroy(h)


def test_batch_cg_converges_per_system():
    specs = [(synth.stencil_3d(14, 13, 12, 27, "random_dd", 7), "f64", 4, (32, 4)),
             (synth.stencil_3d(20, 20, 9, 7, "random_dd", 8), "f64", 1, (32, 8)),
             (synth.fem_like(8, 9), "f32", 2, (32, 2)),
             (synth.stencil_3d(6, 6, 6, 27, "random_dd", 10), "f64", 16, (16, 4))]
    hs, forms = make_batch(specs)
    b = csrk.batch_create(hs, [k for _, _, k, _ in specs])
    Bs = [torch.tensor(synth.uniform_block(a.n, k, 300 + i), device=DEV) for i, (a, _, k, _) in enumerate(specs)]
    Xs = [torch.zeros_like(x) for x in Bs]
    rel, its = csrk.batch_cg(b, Bs, Xs, 200, 1e-10)
    assert np.all(rel <= 1.05e-10), rel
    assert np.all(its > 0) and np.all(its <= 200)
    q = 0
    for i, ((a, _, k, _), (rp, ci, v)) in enumerate(zip(specs, forms)):
        X, B = Xs[i].cpu().numpy(), Bs[i].cpu().numpy()
        for c in range(k):
            r = B[:, c] - ospmv.csr_spmv(a.n, rp, ci, v, X[:, c])
            true = np.linalg.norm(r) / np.linalg.norm(B[:, c])
            assert true <= 1.05e-10 and abs(true - rel[q]) <= 1e-12 + 1e-3 * true
            q += 1
    # a second solve replays the same graph
    rel2, its2 = csrk.batch_cg(b, Bs, Xs, 200, 1e-10)
    assert np.array_equal(its, its2) and np.allclose(rel, rel2, rtol=1e-12, atol=0)
    csrk.batch_destroy(b)
    for h in hs:
        csrk.destroy(h)


def test_batch_rejects_natural_numbering():
    a = synth.stencil_2d_5pt(8, 8)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.set_sizes(h, 8, 2)
    b = csrk.batch_create([h], [1])
    x = torch.zeros(a.n, dtype=torch.float64, device=DEV)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.batch_spmm(b, 1.0, [x], 0.0, [torch.zeros_like(x)], flags=0)
    assert ei.value.status == "ERR_UNSUPPORTED"
    csrk.batch_destroy(b)
    csrk.destroy(h)


SOLVE_SPECS = [(synth.stencil_3d(14, 13, 12, 27, "random_dd", 31), "f64", 4, (32, 4)),
               (synth.stencil_3d(20, 20, 9, 7, "random_dd", 32), "f32", 1, (32, 8)),
               (synth.fem_like(8, 33), "f32", 2, (32, 2)),
               (synth.stencil_3d(6, 6, 6, 27, "random_dd", 34), "f64", 16, (16, 4)),
               (synth.stencil_2d_5pt(17, 13), "bf16", 8, (32, 1))]


def solve_setup(specs):
    hs, forms = [], []
    for a, dtype, k, sizes in specs:
        h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, dtype)
        csrk.reorder(h)
        csrk.set_sizes(h, *sizes)
        e = csrk.export(h)
        forms.append((e["rowptr"], e["colidx"], e["vals"]))   # the FP64 operator
        hs.append(h)
    b = csrk.batch_create(hs, [k for _, _, k, _ in specs])
    Bs = [torch.tensor(synth.uniform_block(a.n, k, 600 + i), device=DEV) for i, (a, _, k, _) in enumerate(specs)]
    return hs, forms, b, Bs


@pytest.mark.parametrize("inner,restart", [("f64", 0), ("f32", 0), ("bf16", 1)])
def test_batch_cg_solve_reaches_rtol_on_the_fp64_operator(inner, restart):
    hs, forms, b, Bs = solve_setup(SOLVE_SPECS)
    Xs = [torch.full_like(x, np.nan) for x in Bs]
    rc, rel, its, cycles = csrk.batch_cg_solve(b, Bs, Xs, rtol=1e-10, maxit=3000, inner=inner, restart=restart)
    assert rc == 0 and cycles >= 1
    assert np.all(rel <= 1e-10), rel
    q = 0
    for i, ((a, _, k, _), (rp, ci, v)) in enumerate(zip(SOLVE_SPECS, forms)):
        X, B = Xs[i].cpu().numpy(), Bs[i].cpu().numpy()
        for c in range(k):
            true = np.linalg.norm(B[:, c] - ospmv.csr_spmv(a.n, rp, ci, v, X[:, c])) / np.linalg.norm(B[:, c])
            assert true <= 1.05e-10 and abs(true - rel[q]) <= 1e-13 + 1e-3 * true, (i, c, true, rel[q])
            if inner == "f64":          # same recurrences, same stopping rule: same count up to rounding
                _, it_ref, _ = ocg.cg_fp64(a.n, rp, ci, v, B[:, c], rtol=1e-10)
                assert abs(int(its[q]) - it_ref) <= 3, (i, c, its[q], it_ref)
            else:                       # the oracle's mixed CG sums the rounded products in FP64
                _, it_ref, res_ref = ocg.cg_mixed(a.n, rp, ci, v, B[:, c], lo=inner, rtol=1e-10,
                                                  replace_every=20, restart=bool(restart))
                assert res_ref <= 1e-10 and abs(int(its[q]) - it_ref) <= max(8, 0.25 * it_ref), (i, c, its[q], it_ref)
            q += 1
    # a second solve replays the cycle graph and reproduces the result exactly
    Xs2 = [torch.zeros_like(x) for x in Bs]
    rc2, rel2, its2, cycles2 = csrk.batch_cg_solve(b, Bs, Xs2, rtol=1e-10, maxit=3000, inner=inner, restart=restart)
    assert rc2 == 0 and cycles2 == cycles and np.array_equal(its, its2) and np.array_equal(rel, rel2)
    assert all(torch.equal(x, y) for x, y in zip(Xs, Xs2))
    assert csrk.batch_device_status(b) == 0
    csrk.batch_destroy(b)
    for h in hs:
        csrk.destroy(h)


def test_batch_cg_solve_matches_oracle_mixed_iterations():
    """One system per matrix: the mixed solve against the oracle's mixed CG (which sums the
    low-precision products in FP64, so counts agree only roughly)."""
    specs = [(synth.stencil_3d(16, 16, 16, 27, "random_dd", 41), "f64", 1, (32, 4)),
             (synth.fem_like(10, 42), "f64", 1, (32, 2))]
    hs, forms, b, Bs = solve_setup(specs)
    Xs = [torch.zeros_like(x) for x in Bs]
    rc, rel, its, _ = csrk.batch_cg_solve(b, Bs, Xs, rtol=1e-10, maxit=3000, inner="f32", restart=1)
    assert rc == 0
    for i, ((a, _, k, _), (rp, ci, v)) in enumerate(zip(specs, forms)):
        B = Bs[i].cpu().numpy()[:, 0]
        _, it_ref, res_ref = ocg.cg_mixed(a.n, rp, ci, v, B, lo="f32", rtol=1e-10, replace_every=20, restart=True)
        assert res_ref <= 1e-10 and abs(int(its[i]) - it_ref) <= max(5, 0.15 * it_ref), (i, its[i], it_ref)
    csrk.batch_destroy(b)
    for h in hs:
        csrk.destroy(h)


def test_batch_cg_solve_iteration_limit_and_fallback(monkeypatch):
    hs, forms, b, Bs = solve_setup(SOLVE_SPECS[:2])
    Xs = [torch.zeros_like(x) for x in Bs]
    rc, rel, its, cycles = csrk.batch_cg_solve(b, Bs, Xs, rtol=1e-10, maxit=20, inner="f64")
    assert rc == 8 and cycles == 1 and np.all(its <= 20) and np.any(rel > 1e-10)   # CSRK_ERR_NOT_CONVERGED
    csrk.batch_destroy(b)
    # the direct-load kernel: FP64 solves run, mixed ones are refused
    monkeypatch.setenv("CSRK_BATCH_ITEM_BYTES", str(1 << 30))
    b = csrk.batch_create(hs, [k for _, _, k, _ in SOLVE_SPECS[:2]])
    assert csrk.batch_plan(b)["stages"] == 0
    rc, rel, _, _ = csrk.batch_cg_solve(b, Bs, Xs, rtol=1e-10, maxit=3000, inner="f64")
    assert rc == 0 and np.all(rel <= 1e-10)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.batch_cg_solve(b, Bs, Xs, inner="f32")
    assert ei.value.status == "ERR_UNSUPPORTED"
    csrk.batch_destroy(b)
    for h in hs:
        csrk.destroy(h)


def test_batch_with_an_empty_matrix():
    specs = [(synth.stencil_3d(9, 8, 7, 7, "random_dd", 70), "f64", 2, (32, 4)),
             (synth.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0)), "f64", 4, (32, 4)),
             (synth.stencil_2d_5pt(11, 9), "f32", 1, (16, 2))]
    hs, forms = make_batch(specs)
    b = csrk.batch_create(hs, [k for _, _, k, _ in specs])
    Xs = [torch.tensor(synth.uniform_block(a.n, k, 71 + i), device=DEV).reshape(a.n, k) for i, (a, _, k, _) in enumerate(specs)]
    Ys = [torch.zeros_like(x) for x in Xs]
    csrk.batch_spmm(b, 1.0, Xs, 0.0, Ys)
    torch.cuda.synchronize()
    for i, ((a, _, k, _), (rp, ci, v)) in enumerate(zip(specs, forms)):
        if a.n == 0:
            continue
        X = Xs[i].cpu().numpy()
        ref = ospmv.csr_spmm(a.n, rp, ci, v, X)
        assert np.allclose(Ys[i].cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    Bs = [torch.tensor(synth.uniform_block(a.n, k, 81 + i), device=DEV).reshape(a.n, k) for i, (a, _, k, _) in enumerate(specs)]
    Xc = [torch.zeros_like(x) for x in Bs]
    rc, rel, its, _ = csrk.batch_cg_solve(b, Bs, Xc, rtol=1e-10, maxit=2000, inner="f32")
    assert rc == 0 and np.all(rel <= 1e-10)
    csrk.batch_destroy(b)
    for h in hs:
        csrk.destroy(h)
