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


def test_static_scratch_refuses_oversized_input():
    one = torch.zeros(4, dtype=torch.int32, device=DEV)
    v = torch.zeros(4, dtype=torch.float64, device=DEV)
    w = torch.zeros(4, dtype=torch.float64, device=DEV)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.spmv_static_scratch(MAX_ROWS + 1, 1, one, one, one, one, v, one, 1.0, v, 0.0, w)
    assert ei.value.status == "ERR_ARG" and "exceeds" in str(ei.value)
