"""GPU parity of kernel 5: each super-super-row's x window staged in shared memory.

Kernel 5 copies the runs of x that an SSR's columns fall in into its shared-memory stage
(TMA bulk copies, plain loads for a last run that ends at n off a 16-byte boundary) and
reads x there through 16-bit window offsets.  It forms the same products in the same
order as kernel 0, so the two agree bit for bit; FP64 results are also held to the
oracle at 1e-12 of sum_j |alpha a_ij x_j| + |beta y_i| (Sec. 1's y = A x, Listing 1's
row loop).
"""
import numpy as np
import pytest

import synth
from oracle import spmv as ospmv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05096_gb300 import csrk  # noqa: E402
from tests.test_gpu_spmv import DEV, assert_close, gpu_spmv, make, narrowed, small_27pt  # noqa: E402


def both_kernels(h, x, unroll=8, warps=16, **kw):
    out = {}
    for kernel in (0, 5):
        csrk.set_config(h, kernel=kernel, lanes=1, unroll=unroll, warps=warps)
        out[kernel] = gpu_spmv(h, x, **kw)
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("unroll", [4, 8, 16])
def test_xwin_bit_exact_with_kernel0(dtype, unroll):
    a = small_27pt(31)
    x = synth.uniform_vector(a.n, 71)
    y0 = synth.uniform_vector(a.n, 72)
    h = make(a, 32, 4, dtype=dtype)
    o1 = both_kernels(h, x, unroll, alpha=1.25, beta=0.5, y0=y0)
    o2 = both_kernels(h, x, unroll)
    assert np.array_equal(o1[0], o1[5]) and np.array_equal(o2[0], o2[5])
    assert_close(o1[5], a, narrowed(a, dtype), x, 1.25, 0.5, y0)
    assert csrk.tuned_config(h)["kernel"] == 5
    csrk.destroy(h)


@pytest.mark.parametrize("dtype,acc_f32", [("f32", False), ("f32", True), ("bf16", True)])
def test_xwin_fp32_vectors(dtype, acc_f32):
    """FP32 x: the window holds 4-byte elements (a run of 4 is one 16-byte copy)."""
    a = small_27pt(33)
    x = synth.uniform_vector(a.n, 73)
    h = make(a, 32, 8, dtype=dtype)
    out = both_kernels(h, x, 8, x_f32=True, acc_f32=acc_f32)
    assert np.array_equal(out[0], out[5])
    x32 = x.astype(np.float32).astype(np.float64)
    if acc_f32:
        m = np.diff(a.rowptr).astype(np.float64)
        assert_close(out[5], a, narrowed(a, dtype), x32, per_row=(m + 3) * 2.0 ** -24)
    else:   # y is stored as FP32: one final rounding on top of the FP64 sum
        assert_close(out[5], a, narrowed(a, dtype), x32, per_row=np.full(a.n, 2.0 ** -24 + 1e-12))
    csrk.destroy(h)


@pytest.mark.parametrize("nx,ny", [(61, 67), (63, 65), (64, 66), (62, 61)])
@pytest.mark.parametrize("x_f32", [False, True])
def test_xwin_ragged_end_of_x(nx, ny, x_f32):
    """n = 4087, 4095, 4224, 3782: the run holding x[n-1] ends at n, off a 16-byte boundary
    for most of these n, so its last elements take the plain-load path."""
    n = nx * ny
    a = synth.stencil_2d_5pt(nx, ny, labels=synth.vectors.permutation(n, 5))
    dtype = "f32" if x_f32 else "f64"
    h = make(a, 32, 8, dtype=dtype)
    x = synth.uniform_vector(n, 74)
    out = both_kernels(h, x, 4, warps=8, x_f32=x_f32, acc_f32=x_f32)
    assert np.array_equal(out[0], out[5])
    if not x_f32:
        assert_close(out[5], a, a.vals, x)
    csrk.destroy(h)


def test_xwin_natural_numbering_and_permuted_vectors():
    """Input-numbering call (permute x, kernel, fused unpermute), CSRK_VEC_PERMUTED vectors,
    and a matrix with no reordering (x is the caller's own tensor)."""
    a = small_27pt(35)
    x = synth.uniform_vector(a.n, 75)
    h = make(a, 32, 4, cfg=dict(kernel=5, lanes=1, unroll=8, warps=8))
    assert_close(gpu_spmv(h, x), a, a.vals, x)
    perm = csrk.export(h)["perm"]
    got_p = gpu_spmv(h, x[perm], flags=csrk.VEC_PERMUTED)
    y = np.empty_like(got_p)
    y[perm] = got_p
    assert_close(y, a, a.vals, x)
    csrk.destroy(h)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.set_sizes(h, 32, 2)
    csrk.set_config(h, kernel=5, lanes=1, unroll=8, warps=8, ctas=1)
    assert_close(gpu_spmv(h, x), a, a.vals, x)
    csrk.destroy(h)


def test_xwin_misaligned_x_refused_when_forced_and_replaced_otherwise():
    """A caller's x 8 bytes off a 16-byte boundary cannot be copied by TMA: a forced kernel 5
    refuses it, a tuned one gives way to another kernel."""
    a = small_27pt(37)
    h = make(a, 32, 4)
    perm = csrk.export(h)["perm"]
    xp = synth.uniform_vector(a.n + 1, 76)
    xt = torch.tensor(xp, device=DEV)[1:]              # x in the reordered numbering, misaligned
    yt = torch.empty(a.n, dtype=torch.float64, device=DEV)
    csrk.set_config(h, kernel=5, lanes=1, unroll=8, warps=8)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.spmv(h, 1.0, xt, 0.0, yt, csrk.VEC_PERMUTED)
    assert ei.value.status == "ERR_UNSUPPORTED"
    csrk.set_sizes(h, 0, 0)                            # tuned, not forced
    csrk.spmv(h, 1.0, xt, 0.0, yt, csrk.VEC_PERMUTED)
    torch.cuda.synchronize()
    assert csrk.device_status(h) == 0
    x = np.empty(a.n)
    x[perm] = xp[1:]                                   # the same x in the input numbering
    y = np.empty(a.n)
    y[perm] = yt.cpu().numpy()
    assert_close(y, a, a.vals, x)
    csrk.destroy(h)


def test_xwin_bandk_pointers_empty_rows_and_long_rows():
    a = synth.random_pattern(3000, 0.002, 77, symmetric=True, empty_rows=200)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder_bandk(h, 16, 3)
    x = synth.uniform_vector(a.n, 78)
    out = both_kernels(h, x, 4, warps=8)
    assert np.array_equal(out[0], out[5])
    assert_close(out[5], a, a.vals, x)
    csrk.destroy(h)
    b = synth.with_dense_rows(small_27pt(39), 3, 4500, 40)
    h = csrk.create(b.n, b.rowptr, b.colidx, b.vals)
    csrk.reorder(h)
    assert csrk.split_long_rows(h, 2048) == 3
    csrk.set_sizes(h, 32, 4)
    x = synth.uniform_vector(b.n, 79)
    y0 = synth.uniform_vector(b.n, 80)
    for kernel in (0, 5):
        csrk.set_config(h, kernel=kernel, lanes=1, unroll=8, warps=8)
        assert_close(gpu_spmv(h, x, 0.5, -1.0, y0), b, b.vals, x, 0.5, -1.0, y0)
    csrk.destroy(h)


def test_xwin_refused_when_windows_do_not_fit():
    """No reordering and large super-super-rows: thousands of scattered columns per SSR,
    windows too large for two shared-memory stages."""
    n = 60 ** 3
    a = synth.stencil_3d(60, 60, 60, 7, "random_dd", 6, labels=synth.vectors.permutation(n, 6))
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.set_sizes(h, 128, 16)
    csrk.set_config(h, kernel=5, lanes=1, unroll=8)
    x = torch.tensor(synth.uniform_vector(n, 81), device=DEV)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.spmv(h, 1.0, x, 0.0, torch.empty_like(x))
    assert ei.value.status == "ERR_UNSUPPORTED"
    csrk.destroy(h)


def test_xwin_spmm_takes_kernel0():
    """SpMM on a handle configured for kernel 5 runs the multi-column kernel."""
    a = small_27pt(41)
    h = make(a, 32, 4, cfg=dict(kernel=5, lanes=1, unroll=8, warps=8))
    X = synth.uniform_block(a.n, 4, 82)
    Xt = torch.tensor(X, device=DEV)
    Yt = torch.empty_like(Xt)
    csrk.spmm(h, 4, 1.0, Xt, 4, 0.0, Yt, 4)
    torch.cuda.synchronize()
    got = Yt.cpu().numpy()
    ref = ospmv.csr_spmm(a.n, a.rowptr, a.colidx, a.vals, X)
    for j in range(4):
        s = ospmv.abs_row_scale(a.rowptr, a.colidx, a.vals, X[:, j].copy())
        assert np.all(np.abs(got[:, j] - ref[:, j]) <= 1e-12 * s)
    csrk.destroy(h)


# ------------------------------------------------------------------ kernel 6: the window with FP32-pair arithmetic
@pytest.mark.parametrize("unroll", [4, 8, 16])
def test_xwin_pairs_fp64_bound(unroll):
    """Kernel 6 keeps FP64 values as (hi, lo) FP32 pairs and row sums as FP32 pairs on the
    FP32 pipes, x from the staged window of its split: within the FP64 bound of the
    oracle (not bit-identical to kernel 0: the arithmetic differs)."""
    for a in (small_27pt(43), synth.fem_like(12, 5), synth.random_pattern(500, 0.03, 15, empty_rows=30)):
        x = synth.uniform_vector(a.n, 83)
        h = make(a, 32, 4, cfg=dict(kernel=6, lanes=1, unroll=unroll, warps=8))
        assert csrk.tuned_config(h)["kernel"] == 6
        assert_close(gpu_spmv(h, x), a, a.vals, x)
        y0 = synth.uniform_vector(a.n, 84)
        assert_close(gpu_spmv(h, x, -0.5, 2.0, y0), a, a.vals, x, -0.5, 2.0, y0)
        perm = csrk.export(h)["perm"]
        got_p = gpu_spmv(h, x[perm], flags=csrk.VEC_PERMUTED)
        y = np.empty_like(got_p)
        y[perm] = got_p
        assert_close(y, a, a.vals, x)
        csrk.destroy(h)


def test_xwin_pairs_integer_exact_and_extreme_x():
    """Integer-valued inputs are exact; zeros, tiny, huge and non-finite x entries make the
    split pass flag the launch, whose window then holds FP64 x and whose products are FP64."""
    a = synth.random_pattern(400, 0.03, 16, integer_values=True, empty_rows=20)
    xi = np.random.default_rng(17).integers(-1000, 1001, size=a.n).astype(np.float64)
    h = make(a, 16, 4, cfg=dict(kernel=6, lanes=1, unroll=8, warps=8))
    assert np.array_equal(gpu_spmv(h, xi), ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, xi))
    x = synth.uniform_vector(a.n, 18)
    x[::7] = 0.0
    x[1::11] = 1e-300
    x[2::13] = 3e150
    x[3::17] = -2.0 ** -45
    assert_close(gpu_spmv(h, x), a, a.vals, x)
    xn = x.copy()
    xn[5] = np.inf
    xn[9] = np.nan
    ref = ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, xn)
    got = gpu_spmv(h, xn)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    fin = np.isfinite(ref)
    assert np.array_equal(got[~fin & ~np.isnan(ref)], ref[~fin & ~np.isnan(ref)])
    csrk.destroy(h)


def test_xwin_pairs_refused_for_out_of_range_values_and_misaligned_x():
    a = synth.stencil_3d(8, 8, 8, 7, "random_dd", 19)
    a.vals[5] = 1e-30
    x = synth.uniform_vector(a.n, 20)
    h = make(a, 32, 4, cfg=dict(kernel=6, lanes=1, unroll=8, warps=8))
    with pytest.raises(csrk.CsrkError) as ei:
        gpu_spmv(h, x)
    assert ei.value.status == "ERR_UNSUPPORTED"
    csrk.destroy(h)
    b = small_27pt(45)
    h = make(b, 32, 4, cfg=dict(kernel=6, lanes=1, unroll=8, warps=8))
    xt = torch.tensor(synth.uniform_vector(b.n + 1, 85), device=DEV)[1:]
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.spmv(h, 1.0, xt, 0.0, torch.empty(b.n, dtype=torch.float64, device=DEV), csrk.VEC_PERMUTED)
    assert ei.value.status == "ERR_UNSUPPORTED"
    csrk.destroy(h)


def test_xwin_pairs_in_cg():
    """FP64 CG on a handle set to kernel 6 (its SpMVs split p each iteration) reaches the
    tolerance by the true residual."""
    a = synth.stencil_3d(24, 23, 22, 27, "random_dd", 46, labels=synth.vectors.permutation(24 * 23 * 22, 46))
    h = make(a, 32, 4, cfg=dict(kernel=6, lanes=1, unroll=8, warps=8))
    b = synth.uniform_vector(a.n, 86)
    bt = torch.tensor(b, device=DEV)
    xt = torch.zeros_like(bt)
    rc, it, rel = csrk.cg(h, bt, xt, 1e-10, 2000, "f64", 20, 0)
    assert rc == 0 and rel <= 1e-10
    true = np.linalg.norm(b - ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, xt.cpu().numpy())) / np.linalg.norm(b)
    assert true <= 1.05e-10
    csrk.destroy(h)


# ------------------------------------------------------------------ length order of irregular rows
@pytest.mark.parametrize("kernel", [5, 6])
def test_xwin_row_length_order(kernel):
    """Rows of unequal length (FEM-like, 13-24 entries; a random pattern with empty rows):
    the window kernels hand each SSR's rows to warp passes in order of length.  Each row's
    arithmetic is unchanged, so kernel 5 stays bit-identical to kernel 0; kernel 6 within
    the FP64 bound."""
    for a in (synth.fem_like(14, 7), synth.random_pattern(4000, 0.004, 87, empty_rows=100)):
        h = make(a, 32, 4)
        info = csrk.xwin_info(h)
        assert info["available"] and info["row_order"]
        x = synth.uniform_vector(a.n, 88)
        y0 = synth.uniform_vector(a.n, 89)
        csrk.set_config(h, kernel=0, lanes=1, unroll=8, warps=8)
        ref = gpu_spmv(h, x, 0.75, -1.5, y0)
        csrk.set_config(h, kernel=kernel, lanes=1, unroll=8, warps=8)
        got = gpu_spmv(h, x, 0.75, -1.5, y0)
        if kernel == 5:
            assert np.array_equal(got, ref)
        assert_close(got, a, a.vals, x, 0.75, -1.5, y0)
        perm = csrk.export(h)["perm"]
        got_p = gpu_spmv(h, x[perm], flags=csrk.VEC_PERMUTED)
        y = np.empty_like(got_p)
        y[perm] = got_p
        assert_close(y, a, a.vals, x)
        csrk.destroy(h)

