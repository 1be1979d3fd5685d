"""GPU parity: the CUDA CSR-k path (through the C ABI) against the FP64 oracle.

Error measure per entry i: |y_gpu - y_ref| / s_i with s_i = |alpha| sum_j |a_ij x_j| +
|beta| |y_i| (rows with s_i = 0 must match exactly).  Bounds:
  FP64 values, FP64 accumulation: 1e-12 (the target of the method's FP64 parity).
  narrowed values (FP32 / BF16) with FP64 accumulation: 1e-12 against the oracle run on the
    same narrowed values (storage rounding is reproduced bit for bit on the host, so only
    the accumulation differs).
  FP32 accumulation with FP32 x: (m_i + 3) * 2^-24 against the oracle on the narrowed
    values and the FP32-rounded x, m_i the row length (one rounding per add, one for the
    products, one each for alpha and beta).
Integer-valued inputs are compared bit for bit.
"""
import numpy as np
import pytest

import synth
from oracle import precision, spmv as ospmv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05096_gb300 import csrk  # noqa: E402

DEV = "cuda:0"


def make(a, sr=32, ssr=8, dtype="f64", method="rcm", cfg=None, pointers=None):
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, dtype)
    csrk.reorder(h, method)
    if pointers is not None:
        csrk.set_pointers(h, *pointers)
    else:
        csrk.set_sizes(h, sr, ssr)
    if cfg:
        csrk.set_config(h, **cfg)
    return h


def narrowed(a, dtype):
    if dtype == "f64":
        return a.vals
    if dtype == "f32":
        return precision.to_f32(a.vals).astype(np.float64)
    return precision.bf16_bits_to_f64(precision.to_bf16_bits(a.vals))


def gpu_spmv(h, x, alpha=1.0, beta=0.0, y0=None, x_f32=False, acc_f32=False, flags=0):
    dt = torch.float32 if x_f32 else torch.float64
    xt = torch.tensor(x, dtype=dt, device=DEV)
    if y0 is None:
        yt = torch.full((x.shape[0],), float("nan"), dtype=dt, device=DEV)
    else:
        yt = torch.tensor(y0, dtype=dt, device=DEV)
    f = flags | (csrk.X_F32 if x_f32 else 0) | (csrk.ACC_F32 if acc_f32 else 0)
    csrk.spmv(h, alpha, xt, beta, yt, f)
    torch.cuda.synchronize()
    assert csrk.device_status(h) == 0
    return yt.double().cpu().numpy()


def assert_close(got, a, vals, x, alpha=1.0, beta=0.0, y0=None, bound=1e-12, per_row=None):
    ref = ospmv.csr_spmv(a.n, a.rowptr, a.colidx, vals, x, alpha, beta, y0)
    s = ospmv.abs_row_scale(a.rowptr, a.colidx, vals, x, alpha, beta, y0)
    err = np.abs(got - ref)
    tol = bound * s if per_row is None else per_row * s
    bad = ~(err <= tol)
    assert not bad.any(), f"{bad.sum()} rows out of bound; worst {np.max(err / np.where(s > 0, s, 1))}"


def small_27pt(seed=3):
    # 20 x 17 x 15 = 5100 rows: several SSR tiles and a ragged tail for sr=32, ssr=8
    return synth.stencil_3d(20, 17, 15, 27, "random_dd", seed, labels=synth.vectors.permutation(5100, seed))


# ------------------------------------------------------------------ 5-point 64x64 Laplacian, CSR-3 (32, 8)
def test_laplacian_5pt_64x64_fp64():
    """2-D 5-point Laplacian 64x64, rows randomly permuted (seed 1) then RCM, CSR-3 with
    SR = 32 rows and SSR = 8 SRs, x ~ U[-1,1] (seed 2), y = Ax."""
    a = synth.stencil_2d_5pt(64, 64, labels=synth.vectors.permutation(4096, 1))
    h = make(a, 32, 8)
    x = synth.uniform_vector(a.n, 2)
    got = gpu_spmv(h, x)
    assert_close(got, a, a.vals, x)
    ones = gpu_spmv(h, np.ones(a.n))
    assert np.array_equal(ones, ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, np.ones(a.n)))
    csrk.destroy(h)


PAIRS = [(1, 4), (1, 8), (1, 16), (1, 32), (2, 8), (2, 16), (4, 8), (8, 8), (32, 4)]
CONFIGS = ([dict(kernel=0, lanes=l, unroll=u, warps=w) for l, u in PAIRS for w in (1, 8)] +
           [dict(kernel=0, lanes=1, unroll=32, warps=w) for w in (4, 16)] +
           [dict(kernel=0, lanes=1, warps=8, stages=2), dict(kernel=0, lanes=1, warps=8, ctas=2),
            dict(kernel=0, lanes=4, warps=3, stages=3)] +
           [dict(kernel=1, lanes=l, unroll=u, warps=w) for l, u in PAIRS for w in (1, 8)])


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_kernel_configs_fp64(cfg):
    a = small_27pt()
    # two blocks per SM halve the shared memory: 256-row 27-point SSRs no longer fit two stages
    h = make(a, 32, 4 if cfg.get("ctas", 1) > 1 else 8, cfg=cfg)
    x = synth.uniform_vector(a.n, 7)
    assert_close(gpu_spmv(h, x), a, a.vals, x)
    csrk.destroy(h)


@pytest.mark.parametrize("sr,ssr", [(1, 1), (7, 3), (32, 8), (64, 2), (100, 1), (5, 40), (32, 64)])
def test_size_sweep_ragged(sr, ssr):
    a = synth.stencil_3d(13, 11, 7, 7, "random_dd", 5, labels=synth.vectors.permutation(1001, 5))
    x = synth.uniform_vector(a.n, 8)
    for kernel in (0, 1):
        h = make(a, sr, ssr, cfg=dict(kernel=kernel))
        assert_close(gpu_spmv(h, x), a, a.vals, x)
        csrk.destroy(h)


def test_integer_values_bit_exact():
    a = synth.random_pattern(700, 0.02, 9, integer_values=True, empty_rows=40)
    x = np.random.default_rng(10).integers(-50, 51, size=a.n).astype(np.float64)
    ref = ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x)
    for cfg in (dict(kernel=0, lanes=1), dict(kernel=0, lanes=8), dict(kernel=1, lanes=4)):
        h = make(a, 16, 4, cfg=cfg)
        assert np.array_equal(gpu_spmv(h, x), ref)
        csrk.destroy(h)


def test_alpha_beta_and_write_only_y():
    a = small_27pt(4)
    x = synth.uniform_vector(a.n, 11)
    y0 = synth.uniform_vector(a.n, 12)
    h = make(a)
    assert_close(gpu_spmv(h, x, 2.5, -0.75, y0), a, a.vals, x, 2.5, -0.75, y0)
    got = gpu_spmv(h, x, -1.0, 0.0, None)            # y starts as NaN, beta == 0
    assert np.all(np.isfinite(got))
    assert_close(got, a, a.vals, x, -1.0)
    csrk.destroy(h)


def test_empty_rows_tiny_and_empty_matrix():
    for a in (synth.random_pattern(50, 0.05, 13, empty_rows=20),
              synth.random_pattern(1, 1.0, 14), synth.random_pattern(3, 0.0, 15)):
        x = synth.uniform_vector(a.n, 16)
        for kernel in (0, 1):
            h = make(a, 4, 2, cfg=dict(kernel=kernel))
            assert_close(gpu_spmv(h, x), a, a.vals, x)
            csrk.destroy(h)
    h = csrk.create(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    csrk.set_sizes(h, 32, 8)
    e = torch.empty(0, dtype=torch.float64, device=DEV)
    csrk.spmv(h, 1.0, e, 0.0, torch.empty(0, dtype=torch.float64, device=DEV))
    csrk.destroy(h)


def test_fig1_explicit_pointers():
    a = synth.random_pattern(9, 0.4, 12)
    x = synth.uniform_vector(9, 13)
    h = make(a, pointers=([0, 2, 5, 7, 9], [0, 2, 4]), method="none")
    got = gpu_spmv(h, x)
    ref3 = ospmv.csr3_spmv(np.array([0, 2, 4]), np.array([0, 2, 5, 7, 9]), a.rowptr, a.colidx, a.vals, x)
    assert np.allclose(got, ref3, rtol=0, atol=1e-14)
    assert_close(got, a, a.vals, x)
    csrk.destroy(h)


def test_variable_pointers_random():
    a = small_27pt(6)
    rng = np.random.default_rng(6)
    cuts = np.sort(rng.choice(np.arange(1, a.n), size=120, replace=False))
    sr_ptr = np.concatenate([[0], cuts, [a.n]])
    nsr = sr_ptr.size - 1
    scuts = np.sort(rng.choice(np.arange(1, nsr), size=60, replace=False))
    ssr_ptr = np.concatenate([[0], scuts, [nsr]])
    x = synth.uniform_vector(a.n, 17)
    for kernel in (0, 1):
        h = make(a, pointers=(sr_ptr, ssr_ptr), cfg=dict(kernel=kernel))
        assert_close(gpu_spmv(h, x), a, a.vals, x)
        csrk.destroy(h)


# ------------------------------------------------------------------ precision variants
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("mode", ["x64acc64", "x32acc64", "x32acc32"])
def test_narrow_values(dtype, mode):
    a = small_27pt(8)
    x = synth.uniform_vector(a.n, 18)
    v = narrowed(a, dtype)
    x_f32 = mode.startswith("x32")
    acc_f32 = mode.endswith("acc32")
    xr = x.astype(np.float32).astype(np.float64) if x_f32 else x
    for lanes in (1, 4):
        h = make(a, 32, 8, dtype=dtype, cfg=dict(lanes=lanes))
        got = gpu_spmv(h, x, x_f32=x_f32, acc_f32=acc_f32)
        if acc_f32:
            m = np.diff(a.rowptr.astype(np.int64)).astype(np.float64)
            assert_close(got, a, v, xr, per_row=(m + 3) * 2.0 ** -24)
        elif x_f32:
            # y is stored as FP32: one final rounding on top of the FP64 sum
            assert_close(got, a, v, xr, per_row=np.full(a.n, 2.0 ** -24 + 1e-12))
        else:
            assert_close(got, a, v, xr)
        csrk.destroy(h)


def test_error_vs_fp64_stated():
    """Per-entry error of the narrowed formats against the FP64 oracle on FP64 values:
    within the format's unit roundoff u = 2^-p for p significant bits (FP32: 2^-24,
    BF16: 2^-8) plus 1e-12, relative to s_i: each stored value moves by at most u times
    itself, so the row sum moves by at most u * s_i."""
    a = small_27pt(9)
    x = synth.uniform_vector(a.n, 19)
    for dtype, bound in (("f32", 2.0 ** -24), ("bf16", 2.0 ** -8)):
        h = make(a, dtype=dtype)
        assert_close(gpu_spmv(h, x), a, a.vals, x, bound=bound + 1e-12)
        csrk.destroy(h)


# ------------------------------------------------------------------ SpMM
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 16, 17, 32, 33, 64])
def test_spmm(k):
    a = small_27pt(10)
    X = synth.uniform_block(a.n, k, 20)
    Y0 = synth.uniform_block(a.n, k, 21)
    ldx, ldy = k + (k % 3), k + 1
    Xp = np.zeros((a.n, ldx)); Xp[:, :k] = X
    Yp = np.zeros((a.n, ldy)); Yp[:, :k] = Y0
    ref = ospmv.csr_spmm(a.n, a.rowptr, a.colidx, a.vals, X, 1.5, 0.5, Y0)
    for kernel in (0, 1):
        h = make(a, 32, 4, cfg=dict(kernel=kernel))
        Xt = torch.tensor(Xp, device=DEV)
        Yt = torch.tensor(Yp, device=DEV)
        csrk.spmm(h, k, 1.5, Xt, ldx, 0.5, Yt, ldy)
        torch.cuda.synchronize()
        got = Yt.cpu().numpy()
        for c in range(k):
            s = ospmv.abs_row_scale(a.rowptr, a.colidx, a.vals, X[:, c], 1.5, 0.5, Y0[:, c])
            assert np.all(np.abs(got[:, c] - ref[:, c]) <= 1e-12 * s)
        assert np.array_equal(got[:, k:], Yp[:, k:])      # padding columns untouched
        csrk.destroy(h)


# ------------------------------------------------------------------ numbering / host vectors
def test_vec_permuted_and_permute_entry_point():
    a = small_27pt(11)
    x = synth.uniform_vector(a.n, 22)
    h = make(a)
    perm = csrk.export(h)["perm"]
    y_nat = gpu_spmv(h, x)
    xt = torch.tensor(x, device=DEV)
    xp = torch.empty_like(xt)
    csrk.permute(h, 0, 1, xt, 1, xp, 1)
    torch.cuda.synchronize()
    assert np.array_equal(xp.cpu().numpy(), x[perm])
    yp = torch.empty_like(xt)
    csrk.spmv(h, 1.0, xp, 0.0, yp, csrk.VEC_PERMUTED)
    y2 = torch.empty_like(xt)
    csrk.permute(h, 1, 1, yp, 1, y2, 1)
    torch.cuda.synchronize()
    assert np.array_equal(y2.cpu().numpy(), y_nat)
    csrk.destroy(h)


@pytest.mark.parametrize("dims", [(6, 6, 6), (5, 5, 1), (7, 7, 2), (3, 3, 3), (3, 1, 1)])   # n % 4 = 0, 1, 2, 3; n < 4
def test_permute_paths_bit_exact(dims):
    """Gather and scatter through the quad kernel (aligned unit stride), the element-wise
    kernel (a view 8 bytes off a 16-byte boundary) and the k > 1 kernel."""
    nx, ny, nz = dims
    side = nx * ny * nz
    a = synth.stencil_3d(nx, ny, nz, 7, "random_dd", side, labels=synth.vectors.permutation(side, side))
    h = make(a)
    perm = csrk.export(h)["perm"]
    n = a.n
    x = synth.uniform_vector(n + 1, 40 + side)
    base = torch.tensor(x, device=DEV)
    for xt in (base[:n], base[1:]):                    # 16-byte aligned, then 8-byte aligned
        xv = xt.cpu().numpy()
        outb = torch.full((n + 1,), np.nan, dtype=torch.float64, device=DEV)
        for out in (outb[:n], outb[1:]):
            csrk.permute(h, 0, 1, xt, 1, out, 1)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), xv[perm])
            csrk.permute(h, 1, 1, xt, 1, out, 1)
            torch.cuda.synchronize()
            back = np.empty(n)
            back[perm] = xv
            assert np.array_equal(out.cpu().numpy(), back)
    X = synth.uniform_block(n, 5, 50 + side)
    Xt = torch.tensor(X, device=DEV)
    Yt = torch.full((n, 5), np.nan, dtype=torch.float64, device=DEV)
    csrk.permute(h, 0, 3, Xt, 5, Yt, 5)               # k = 3 of ld 5
    torch.cuda.synchronize()
    got = Yt.cpu().numpy()
    assert np.array_equal(got[:, :3], X[perm, :3]) and np.isnan(got[:, 3:]).all()
    csrk.destroy(h)


def test_x_permuted_flag_scatters_y():
    a = small_27pt(15)
    x = synth.uniform_vector(a.n, 28)
    y0 = synth.uniform_vector(a.n, 29)
    h = make(a)
    perm = csrk.export(h)["perm"]
    for kernel in (0, 1):
        csrk.set_config(h, kernel=kernel)
        xp = torch.tensor(x[perm], device=DEV)
        yt = torch.tensor(y0, device=DEV)
        csrk.spmv(h, 1.25, xp, -2.0, yt, csrk.X_PERMUTED)
        torch.cuda.synchronize()
        assert_close(yt.cpu().numpy(), a, a.vals, x, 1.25, -2.0, y0)
    csrk.destroy(h)


def test_host_vectors():
    a = small_27pt(12)
    x = synth.uniform_vector(a.n, 23)
    y0 = synth.uniform_vector(a.n, 24)
    h = make(a)
    y = y0.copy()
    csrk.spmv(h, 0.5, x, 2.0, y, csrk.HOST_VECTORS, stream=0)
    assert_close(y, a, a.vals, x, 0.5, 2.0, y0)
    csrk.destroy(h)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_host_vectors_page_locked(dtype):
    """Page-locked host x is permuted straight from host memory (one pass, through the
    inverse permutation): bit-identical to pageable host vectors and to device vectors,
    for SpMV (beta = 0 and beta != 0) and for SpMM with a padded leading dimension."""
    a = small_27pt(13)
    x = synth.uniform_vector(a.n, 31)
    y0 = synth.uniform_vector(a.n, 32)
    h = make(a, 32, 4, dtype=dtype)
    ref = gpu_spmv(h, x, 0.75, -1.5, y0)
    assert_close(ref, a, narrowed(a, dtype), x, 0.75, -1.5, y0)
    for beta in (0.0, -1.5):
        want = gpu_spmv(h, x, 0.75, beta, y0)
        yp = y0.copy()                                       # pageable host vectors
        csrk.spmv(h, 0.75, x, beta, yp, csrk.HOST_VECTORS, stream=0)
        xt = torch.tensor(x).pin_memory()                    # page-locked host vectors
        yt = torch.tensor(y0).pin_memory()
        csrk.spmv(h, 0.75, xt, beta, yt, csrk.HOST_VECTORS, stream=0)
        assert np.array_equal(yp, want) and np.array_equal(yt.numpy(), want)
    k, ld = 3, 4
    X = synth.uniform_vector(a.n * ld, 33).reshape(a.n, ld)
    Xd = torch.tensor(X, device=DEV)
    Yd = torch.zeros((a.n, ld), dtype=torch.float64, device=DEV)
    csrk.spmm(h, k, 1.0, Xd, ld, 0.0, Yd, ld)
    torch.cuda.synchronize()
    Xh = torch.tensor(X).pin_memory()
    Yh = torch.zeros((a.n, ld), dtype=torch.float64).pin_memory()
    csrk.spmm(h, k, 1.0, Xh, ld, 0.0, Yh, ld, csrk.HOST_VECTORS, stream=0)
    assert np.array_equal(Yh.numpy()[:, :k], Yd.cpu().numpy()[:, :k])
    assert csrk.device_status(h) == 0
    csrk.destroy(h)


# ------------------------------------------------------------------ full size
def _full_stencil(points):
    n = 128 ** 3
    return synth.stencil_3d(128, 128, 128, points, "random_dd", 3, labels=synth.vectors.permutation(n, 3))


@pytest.fixture(scope="module")
def stencils128():
    return {p: _full_stencil(p) for p in (7, 27)}


def assert_every_row(got, a, x, what):
    ref = ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x)
    s = ospmv.abs_row_scale(a.rowptr, a.colidx, a.vals, x)
    bad = ~(np.abs(got - ref) <= 1e-12 * s)
    assert not bad.any(), f"{what}: {bad.sum()} rows out of bound, first {np.flatnonzero(bad)[:5]}"


# Launch shapes of the benchmark's timed 128^3 runs (the autotuner's picks on GB300), each
# pinned here, and the autotuner's own pick on the test's device.
FULL_SHAPES = [
    (7, (32, 8), dict(kernel=4, lanes=1, unroll=16, warps=16, stages=5, ctas=2)),
    (27, (32, 4), dict(kernel=4, lanes=1, unroll=8, warps=8, ctas=2)),
    (7, (32, 8), dict(kernel=5, lanes=1, unroll=8, warps=16, ctas=2)),
    (7, (32, 8), dict(kernel=5, lanes=1, unroll=4, warps=16, ctas=2)),
    (27, (32, 4), dict(kernel=5, lanes=1, unroll=8, warps=8, ctas=2)),
    (27, (32, 2), dict(kernel=5, lanes=1, unroll=8, warps=16, ctas=2)),
    (7, (32, 8), dict(kernel=0, lanes=1, unroll=8, warps=16)),
    (7, "auto", None),
    (27, "auto", None),
]


@pytest.mark.parametrize("points,sizes,cfg", FULL_SHAPES)
def test_full_size_128cubed(stencils128, points, sizes, cfg):
    """128^3 stencils in the benchmark's natural-numbering call (permute x, CSR-3 kernel with
    the fused unpermute): every row against the oracle."""
    a = stencils128[points]
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, "f64")
    csrk.reorder(h)
    if sizes == "auto":
        csrk.set_sizes(h, 0, 0)
    else:
        csrk.set_sizes(h, *sizes)
        csrk.set_config(h, **cfg)
    x = synth.uniform_vector(a.n, 2)
    got = gpu_spmv(h, x)
    assert_every_row(got, a, x, f"{points}-point {sizes} {csrk.tuned_config(h)}")
    csrk.destroy(h)


@pytest.mark.parametrize("points", [7, 27])
def test_full_size_128cubed_laplacian_closed_form(points):
    """The Laplacian's row sums on every row: 0 inside, the count of missing neighbours at
    the boundary (exact in any summation order: small integers)."""
    n = 128 ** 3
    lap = synth.stencil_3d(128, 128, 128, points, "laplacian", labels=synth.vectors.permutation(n, 3))
    h = make(lap, 32, 8)
    ones = gpu_spmv(h, np.ones(lap.n))
    assert np.array_equal(ones, ospmv.csr_spmv(lap.n, lap.rowptr, lap.colidx, lap.vals, np.ones(lap.n)))
    csrk.destroy(h)


# ------------------------------------------------------------------ autotuner
def test_autotuner_picks_a_working_config():
    a = small_27pt(13)
    x = synth.uniform_vector(a.n, 25)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder(h)
    csrk.set_sizes(h, 0, 0)
    inf = csrk.info(h)
    cfg = csrk.tuned_config(h)
    assert inf["sr"] > 0 and inf["ssr"] > 0 and inf["nssr"] > 0
    # on a matrix this small every shape is launch-bound: any timed candidate may win
    assert 0 <= cfg["kernel"] <= 6 and cfg["warps"] in (4, 6, 8, 16) and 1 <= cfg["ctas"] <= 4
    assert_close(gpu_spmv(h, x), a, a.vals, x)
    # a second handle with the same shape reuses the cached choice
    h2 = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder(h2)
    csrk.set_sizes(h2, 0, 0)
    assert csrk.tuned_config(h2) == cfg and csrk.info(h2)["sr"] == inf["sr"]
    csrk.destroy(h)
    csrk.destroy(h2)


_TUNE_CHILD = '''
import sys
sys.path.insert(0, sys.argv[1])
import synth
from paper_2203_05096_gb300 import csrk
a = synth.stencil_3d(20, 18, 16, 7, "random_dd", 3)
h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
csrk.reorder(h)
csrk.set_sizes(h, 0, 0)
inf = csrk.info(h)
print(sorted(csrk.tuned_config(h).items()), inf["sr"], inf["ssr"])
'''


def test_tune_cache_file_reused_across_processes(tmp_path):
    """CSRK_TUNE_CACHE: the first process tunes and appends one line (a whitespace-free
    key and the choice); a second process finds it, installs the same choice and appends
    nothing (it does not tune again)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, CSRK_TUNE_CACHE=str(cache))
    runs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", _TUNE_CHILD, root], env=env, capture_output=True, text=True,
                           timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        runs.append((r.stdout, cache.read_text().splitlines()))
    (out1, lines1), (out2, lines2) = runs
    assert len(lines1) == 1 and len(lines1[0].split()) == 10
    assert lines2 == lines1 and out2 == out1


# ------------------------------------------------------------------ FP64 on FP32 pipes
@pytest.mark.parametrize("kernel,unroll", [(2, 4), (2, 8), (2, 16), (3, 4), (3, 8)])
def test_pair_path_fp64_bound(kernel, unroll):
    for a in (small_27pt(14), synth.fem_like(12, 5),
              synth.random_pattern(500, 0.03, 15, empty_rows=30)):
        x = synth.uniform_vector(a.n, 26)
        h = make(a, 32, 4, cfg=dict(kernel=kernel, lanes=1, unroll=unroll))
        assert csrk.tuned_config(h)["kernel"] == kernel
        assert_close(gpu_spmv(h, x), a, a.vals, x)
        y0 = synth.uniform_vector(a.n, 27)
        assert_close(gpu_spmv(h, x, -0.5, 2.0, y0), a, a.vals, x, -0.5, 2.0, y0)
        csrk.destroy(h)


def test_pair_path_integer_exact_and_extreme_x():
    a = synth.random_pattern(400, 0.03, 16, integer_values=True, empty_rows=20)
    xi = np.random.default_rng(17).integers(-1000, 1001, size=a.n).astype(np.float64)
    h = make(a, 16, 4, cfg=dict(kernel=2, lanes=1, unroll=8))
    assert np.array_equal(gpu_spmv(h, xi), ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, xi))
    # zeros, tiny, huge and non-finite entries go through the per-element FP64 product
    x = synth.uniform_vector(a.n, 18)
    x[::7] = 0.0
    x[1::11] = 1e-300
    x[2::13] = 3e150
    x[3::17] = -2.0 ** -45
    got = gpu_spmv(h, x)
    assert_close(got, a, a.vals, x)
    xn = x.copy()
    xn[5] = np.inf
    xn[9] = np.nan
    ref = ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, xn)
    got = gpu_spmv(h, xn)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    fin = np.isfinite(ref)
    assert np.array_equal(got[~fin & ~np.isnan(ref)], ref[~fin & ~np.isnan(ref)])
    csrk.destroy(h)


def test_pair_path_refused_for_out_of_range_values():
    a = synth.stencil_3d(8, 8, 8, 7, "random_dd", 19)
    a.vals[5] = 1e-30                      # below 2^-39: the pair arithmetic would lose accuracy
    x = synth.uniform_vector(a.n, 20)
    h = make(a, 32, 4, cfg=dict(kernel=2, lanes=1, unroll=8))
    with pytest.raises(csrk.CsrkError) as ei:
        gpu_spmv(h, x)
    assert ei.value.status == "ERR_UNSUPPORTED"
    csrk.set_config(h, kernel=0)
    assert_close(gpu_spmv(h, x), a, a.vals, x)
    csrk.destroy(h)


# ------------------------------------------------------------------ Band-k pointers
BANDK_GPU = [
    ("stencil27", lambda: small_27pt(17), (32, 4)),
    ("stencil7", lambda: synth.stencil_3d(30, 20, 11, 7, "random_dd", 18, labels=synth.vectors.permutation(6600, 18)), (32, 8)),
    ("fem", lambda: synth.fem_like(12, 19), (16, 3)),
    ("random", lambda: synth.random_pattern(3000, 0.003, 20, symmetric=True, empty_rows=25), (8, 5)),
]


@pytest.mark.parametrize("name,make,caps", BANDK_GPU, ids=[c[0] for c in BANDK_GPU])
@pytest.mark.parametrize("kernel", [0, 1])
def test_bandk_pointers_spmv(name, make, caps, kernel):
    """Variable super-rows and super-super-rows from Band-k, natural-numbering SpMV (fused
    unpermute) and the reordered-numbering form, TMA-staged and direct-load kernels."""
    a = make()
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    perm = csrk.reorder_bandk(h, *caps)
    csrk.set_config(h, kernel=kernel, lanes=1, unroll=8, warps=8)
    x = synth.uniform_vector(a.n, 31)
    y0 = synth.uniform_vector(a.n, 32)
    assert_close(gpu_spmv(h, x, 1.5, -0.25, y0), a, a.vals, x, 1.5, -0.25, y0)
    e = csrk.export(h)
    b = synth.CSR(a.n, e["rowptr"], e["colidx"], e["vals"])
    assert_close(gpu_spmv(h, x[perm], flags=csrk.VEC_PERMUTED), b, b.vals, x[perm])
    csrk.destroy(h)


def test_bandk_autotune_keeps_pointers():
    a = small_27pt(21)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder_bandk(h, 32, 4)
    before = csrk.export(h)
    csrk.set_sizes(h, 0, 0)
    after = csrk.export(h)
    assert np.array_equal(before["sr_ptr"], after["sr_ptr"]) and np.array_equal(before["ssr_ptr"], after["ssr_ptr"])
    assert csrk.info(h)["sr"] == 0
    x = synth.uniform_vector(a.n, 33)
    assert_close(gpu_spmv(h, x), a, a.vals, x)
    csrk.set_sizes(h, 32, 8)                          # explicit sizes replace them; the order stays
    assert np.array_equal(csrk.export(h)["perm"], before["perm"]) and csrk.info(h)["sr"] == 32
    assert_close(gpu_spmv(h, x), a, a.vals, x)
    csrk.destroy(h)


# ------------------------------------------------------------------ 16-bit column offsets
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("unroll", [4, 8, 16])
def test_col16_kernel_bit_exact_with_kernel0(dtype, unroll):
    """Kernel 4 reads 16-bit column offsets from each SSR's smallest column; the products
    and their order are kernel 0's, so the results are bit-identical."""
    a = small_27pt(23)
    x = synth.uniform_vector(a.n, 41)
    y0 = synth.uniform_vector(a.n, 42)
    h = make(a, 32, 4, dtype=dtype)
    assert csrk.index_bits(h) == 16
    out = {}
    for kernel in (0, 4):
        csrk.set_config(h, kernel=kernel, lanes=1, unroll=unroll, warps=16)
        out[kernel] = (gpu_spmv(h, x, 1.25, 0.5, y0), gpu_spmv(h, x))
    assert np.array_equal(out[0][0], out[4][0]) and np.array_equal(out[0][1], out[4][1])
    if dtype == "f64":
        assert_close(out[4][0], a, a.vals, x, 1.25, 0.5, y0)
    csrk.destroy(h)


def test_col16_full_size_27pt_fused_unpermute(stencils128):
    a = stencils128[27]
    h = make(a, 32, 2)
    assert csrk.index_bits(h) == 16
    csrk.set_config(h, kernel=4, lanes=1, unroll=16, warps=16, ctas=2)
    x = synth.uniform_vector(a.n, 43)
    got = gpu_spmv(h, x)
    assert_every_row(got, a, x, "kernel 4 (32, 2)")
    csrk.set_config(h, kernel=0)
    assert np.array_equal(gpu_spmv(h, x), got)
    csrk.destroy(h)


def test_col16_refused_when_the_span_is_too_wide():
    a = synth.stencil_3d(50, 50, 50, 7, "random_dd", 4, labels=synth.vectors.permutation(125000, 4))
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.set_sizes(h, 32, 8)                          # no reordering: spans of ~125K columns
    assert csrk.index_bits(h) == 32
    csrk.set_config(h, kernel=4, lanes=1, unroll=8)
    x = torch.tensor(synth.uniform_vector(a.n, 44), device=DEV)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.spmv(h, 1.0, x, 0.0, torch.empty_like(x))
    assert ei.value.status == "ERR_UNSUPPORTED"
    csrk.set_sizes(h, 0, 0)                           # the autotuner never picks it here
    assert csrk.tuned_config(h)["kernel"] != 4
    got = gpu_spmv(h, x.cpu().numpy())
    assert_close(got, a, a.vals, x.cpu().numpy())
    csrk.destroy(h)


# ------------------------------------------------------------------ long rows
def long_row_matrix():
    # 5,100-row 27-point stencil plus three coupling rows of ~4,500 entries each (three
    # segments of 2,048), under the stencil's random labelling
    return synth.with_dense_rows(small_27pt(29), 3, 4500, 30)


@pytest.mark.parametrize("dtype,kernel", [("f64", 0), ("f64", 1), ("f64", 2), ("f64", 4), ("f32", 0), ("bf16", 4)])
def test_long_rows_spmv(dtype, kernel):
    a = long_row_matrix()
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, dtype)
    csrk.reorder(h)
    assert csrk.split_long_rows(h, 1000) == 3
    csrk.set_sizes(h, 32, 4)
    csrk.set_config(h, kernel=kernel, lanes=1, unroll=8)
    vals = {"f64": a.vals, "f32": precision.to_f32(a.vals).astype(np.float64),
            "bf16": precision.bf16_bits_to_f64(precision.to_bf16_bits(a.vals))}[dtype]
    bound = 1e-12   # against the oracle on the stored (rounded) values
    x = synth.uniform_vector(a.n, 51)
    y0 = synth.uniform_vector(a.n, 52)
    assert_close(gpu_spmv(h, x, 0.75, -1.5, y0), a, vals, x, 0.75, -1.5, y0, bound=bound)
    if dtype != "f64":   # FP32 vectors and accumulation
        got = gpu_spmv(h, x.astype(np.float32).astype(np.float64), x_f32=True, acc_f32=True)
        assert_close(got, a, vals, x.astype(np.float32).astype(np.float64), bound=(np.max(a.row_lengths()) + 2) * 2.0 ** -24)
    csrk.destroy(h)


@pytest.mark.parametrize("k", [2, 5])
def test_long_rows_spmm(k):
    a = long_row_matrix()
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder(h)
    csrk.split_long_rows(h, 1000)
    csrk.set_sizes(h, 32, 4)
    X = synth.uniform_block(a.n, k, 53)
    Y0 = synth.uniform_block(a.n, k, 54)
    Xt, Yt = torch.tensor(X, device=DEV), torch.tensor(Y0, device=DEV)
    csrk.spmm(h, k, 1.5, Xt, k, 0.5, Yt, k)
    torch.cuda.synchronize()
    ref = ospmv.csr_spmm(a.n, a.rowptr, a.colidx, a.vals, X, 1.5, 0.5, Y0)
    got = Yt.cpu().numpy()
    for c in range(k):
        s = ospmv.abs_row_scale(a.rowptr, a.colidx, a.vals, X[:, c], 1.5, 0.5, Y0[:, c])
        assert np.all(np.abs(got[:, c] - ref[:, c]) <= 1e-12 * s)
    csrk.destroy(h)


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_long_rows_cg_and_autotune(inner):
    a = long_row_matrix()
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder(h)
    csrk.split_long_rows(h, 1000)
    csrk.set_sizes(h, 0, 0)                                  # the autotuner times the long rows too
    b = synth.uniform_vector(a.n, 55)
    bt = torch.tensor(b, device=DEV)
    xt = torch.zeros_like(bt)
    rc, iters, rel = csrk.cg(h, bt, xt, 1e-10, 3000, inner, 20, 0)
    assert rc == 0 and rel <= 1e-10
    r = b - ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, xt.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.05e-10
    with pytest.raises(csrk.CsrkError) as ei:                # batches take no split rows
        csrk.batch_create([h], [1])
    assert ei.value.status == "ERR_UNSUPPORTED"
    csrk.destroy(h)


# ------------------------------------------------------------------ degenerate shapes of the newer paths
def test_col16_with_bandk_pointers_and_empty_rows():
    a = synth.random_pattern(3000, 0.002, 61, symmetric=True, empty_rows=200)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder_bandk(h, 16, 3)
    assert csrk.index_bits(h) == 16
    x = synth.uniform_vector(a.n, 62)
    out = []
    for kernel in (0, 4):
        csrk.set_config(h, kernel=kernel, lanes=1, unroll=4, warps=8)
        out.append(gpu_spmv(h, x))
    assert np.array_equal(out[0], out[1])
    assert_close(out[1], a, a.vals, x)
    csrk.destroy(h)


@pytest.mark.parametrize("lengths", [(2048, 2049, 4096), (1, 1, 1)])
def test_long_rows_segment_boundaries_and_all_rows_long(lengths):
    """Rows of exactly one segment, one entry over, two full segments; and a threshold of
    1 that moves every row out of the super-rows (no SSR at all)."""
    rng = np.random.default_rng(63)
    n = 5000
    rows = [sorted(set([i] + rng.choice(n, 3, replace=False).tolist())) for i in range(n)]
    for r, L in zip((7, 1234, 4999), lengths):
        if L > 1:
            rows[r] = sorted(set([r] + rng.choice(n, L - 1, replace=False).tolist()))
            while len(rows[r]) < L:
                rows[r] = sorted(set(rows[r] + rng.choice(n, L - len(rows[r]), replace=False).tolist()))
    rp = np.array([0] + np.cumsum([len(r) for r in rows]).tolist(), np.int32)
    ci = np.array([c for r in rows for c in r], np.int32)
    vals = rng.standard_normal(ci.size)
    a = synth.CSR(n, rp, ci, vals)
    h = csrk.create(n, rp, ci, vals)
    thr = 2048 if lengths[0] > 1 else 1
    nl = csrk.split_long_rows(h, thr)
    assert nl == (3 if thr > 1 else n)
    csrk.set_sizes(h, 32, 4)
    assert csrk.info(h)["nssr"] == (0 if thr == 1 else csrk.info(h)["nssr"])
    x = synth.uniform_vector(n, 64)
    y0 = synth.uniform_vector(n, 65)
    assert_close(gpu_spmv(h, x, -1.0, 2.0, y0), a, vals, x, -1.0, 2.0, y0)
    csrk.destroy(h)
