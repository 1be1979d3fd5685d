"""csrk_spmv_static_scratch: the allocation-free SpMV entry point.

Some callers cannot let a library allocate device memory -- their arena allocator owns
the GPU, their host program gives them a fixed budget, or an allocation's device
synchronisation would break a latency-critical loop.  This entry point serves them with
a static device scratch array instead of cudaMalloc.  The test checks it against the
regular csrk_spmv (which allocates its scratch) on two calls in a row, through the C
ABI, within the FP64 parity bound used by the other GPU tests (1e-12 of
sum_j |alpha a_ij x_j| + |beta y_i| per entry), and that oversized inputs are refused.
It lives in its own file, collected last, so that a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest

import synth
from oracle import spmv as ospmv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05096_gb300 import csrk  # noqa: E402

DEV = "cuda:0"
MAX_ROWS = 1 << 20


def _device_form(h):
    e = csrk.export(h)
    d = {k: torch.tensor(e[k], device=DEV) for k in ("perm", "rowptr", "colidx", "vals", "sr_ptr", "ssr_ptr")}
    return d, e


def test_static_scratch_matches_spmv_on_two_calls():
    n = 40 * 37 * 31
    a = synth.stencil_3d(40, 37, 31, 27, "random_dd", 3, labels=synth.vectors.permutation(n, 3))
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, "f64")
    csrk.reorder(h, "rcm")
    csrk.set_sizes(h, 32, 8)
    d, e = _device_form(h)
    nssr = e["ssr_ptr"].size - 1
    for call, (alpha, beta) in enumerate(((1.0, 0.0), (1.5, -0.5))):
        x = synth.uniform_vector(n, 100 + call)
        y0 = synth.uniform_vector(n, 200 + call)
        xt = torch.tensor(x, device=DEV)
        ref_t = torch.tensor(y0, device=DEV)
        csrk.spmv(h, alpha, xt, beta, ref_t)
        got_t = torch.tensor(y0, device=DEV)
        csrk.spmv_static_scratch(n, nssr, d["ssr_ptr"], d["sr_ptr"], d["rowptr"], d["colidx"], d["vals"],
                                 d["perm"], alpha, xt, beta, got_t)
        torch.cuda.synchronize()
        ref, got = ref_t.cpu().numpy(), got_t.cpu().numpy()
        scale = ospmv.abs_row_scale(a.rowptr, a.colidx, a.vals, x, alpha, beta, y0)
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), f"call {call}"
        oracle = ospmv.csr_spmv(n, a.rowptr, a.colidx, a.vals, x, alpha, beta, y0)
        assert np.all(np.abs(got - oracle) <= 1e-12 * scale), f"call {call} vs oracle"
    csrk.destroy(h)


def _natural_csr3(a, sr=32, ssr=4, long_min=0):
    """A handle without reordering (optionally with long rows split off) and the device form
    its export gives; the export's permutation is the one csrk_split_long_rows made, or the
    identity."""
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, "f64")
    if long_min:
        csrk.split_long_rows(h, long_min)
    csrk.set_sizes(h, sr, ssr)
    return (h,) + _device_form(h)


def test_static_scratch_without_permutation():
    """perm = NULL: the kernels work on the caller's x and y in place of the static array."""
    a = synth.stencil_3d(30, 29, 31, 7, "random_dd", 5)
    n = a.n
    h, d, e = _natural_csr3(a)
    assert np.array_equal(e["perm"], np.arange(n))
    x = synth.uniform_vector(n, 301)
    y0 = synth.uniform_vector(n, 302)
    for alpha, beta in ((1.0, 0.0), (-0.75, 2.0)):
        got_t = torch.tensor(y0, device=DEV)
        csrk.spmv_static_scratch(n, e["ssr_ptr"].size - 1, d["ssr_ptr"], d["sr_ptr"], d["rowptr"], d["colidx"],
                                 d["vals"], None, alpha, torch.tensor(x, device=DEV), beta, got_t)
        torch.cuda.synchronize()
        ref = ospmv.csr_spmv(n, a.rowptr, a.colidx, a.vals, x, alpha, beta, y0)
        scale = ospmv.abs_row_scale(a.rowptr, a.colidx, a.vals, x, alpha, beta, y0)
        assert np.all(np.abs(got_t.cpu().numpy() - ref) <= 1e-12 * scale)
    xt = torch.tensor(x, device=DEV)
    with pytest.raises(csrk.CsrkError) as ei:        # overlapping x and y without a permutation
        csrk.spmv_static_scratch(n - 1, e["ssr_ptr"].size - 1, d["ssr_ptr"], d["sr_ptr"], d["rowptr"],
                                 d["colidx"], d["vals"], None, 1.0, xt[:-1], 0.0, xt[1:])
    assert ei.value.status == "ERR_ARG"
    csrk.destroy(h)


def test_static_scratch_long_rows_are_computed():
    """After csrk_split_long_rows the export's super-rows end before the long rows; the
    entry point computes those rows too (every entry of y checked)."""
    base = synth.stencil_3d(20, 17, 15, 27, "random_dd", 7, labels=synth.vectors.permutation(5100, 7))
    a = synth.with_dense_rows(base, 3, 4500, 8)
    h, d, e = _natural_csr3(a, long_min=2048)
    n = a.n
    nsr_cover = e["sr_ptr"][-1]
    assert nsr_cover == n - 3                        # three rows after the last super-row
    x = synth.uniform_vector(n, 303)
    y0 = synth.uniform_vector(n, 304)
    got_t = torch.tensor(y0, device=DEV)
    csrk.spmv_static_scratch(n, e["ssr_ptr"].size - 1, d["ssr_ptr"], d["sr_ptr"], d["rowptr"], d["colidx"],
                             d["vals"], d["perm"], 0.5, torch.tensor(x, device=DEV), -1.0, got_t)
    torch.cuda.synchronize()
    ref = ospmv.csr_spmv(n, a.rowptr, a.colidx, a.vals, x, 0.5, -1.0, y0)
    scale = ospmv.abs_row_scale(a.rowptr, a.colidx, a.vals, x, 0.5, -1.0, y0)
    assert np.all(np.abs(got_t.cpu().numpy() - ref) <= 1e-12 * scale)
    csrk.destroy(h)


def test_static_scratch_allocates_nothing_and_allows_aliasing_with_perm():
    """After a first call (which may load the library's device code and its static array),
    further calls leave the device's free memory unchanged; with a permutation x and y may
    be one vector."""
    a = synth.stencil_3d(24, 25, 26, 27, "random_dd", 9, labels=synth.vectors.permutation(24 * 25 * 26, 9))
    n = a.n
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, "f64")
    csrk.reorder(h, "rcm")
    csrk.set_sizes(h, 32, 4)
    d, e = _device_form(h)
    nssr = e["ssr_ptr"].size - 1
    x = synth.uniform_vector(n, 305)
    xt = torch.tensor(x, device=DEV)
    yt = torch.empty_like(xt)
    args = (n, nssr, d["ssr_ptr"], d["sr_ptr"], d["rowptr"], d["colidx"], d["vals"], d["perm"])
    csrk.spmv_static_scratch(*args, 1.0, xt, 0.0, yt)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        csrk.spmv_static_scratch(*args, 1.0, xt, 0.0, yt)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    inout = xt.clone()
    csrk.spmv_static_scratch(*args, 1.0, inout, 0.0, inout)   # y = A y in place
    torch.cuda.synchronize()
    assert torch.equal(inout, yt)
    csrk.destroy(h)


def test_static_scratch_refuses_oversized_input():
    one = torch.zeros(4, dtype=torch.int32, device=DEV)
    v = torch.zeros(4, dtype=torch.float64, device=DEV)
    w = torch.zeros(4, dtype=torch.float64, device=DEV)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.spmv_static_scratch(MAX_ROWS + 1, 1, one, one, one, one, v, one, 1.0, v, 0.0, w)
    assert ei.value.status == "ERR_ARG" and "exceeds" in str(ei.value)
