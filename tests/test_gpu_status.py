"""Device-side failure detection without a GPU fault: a bounded wait that nothing completes
gives up, reports through the status word, and the context stays usable."""
import numpy as np
import pytest

import synth
from oracle import spmv as ospmv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05096_gb300 import csrk  # noqa: E402


def test_bounded_wait_times_out_and_context_survives():
    a = synth.stencil_3d(10, 10, 10, 7, "random_dd", 1)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder(h)
    csrk.set_sizes(h, 32, 4)
    rc, word = csrk.selftest_bounded_wait(h, 20_000_000)      # 20 ms
    assert rc == 7 and word == 1                              # CSRK_ERR_TIMEOUT, bit 0
    assert csrk.device_status(h) == 0                         # the word was cleared
    x = synth.uniform_vector(a.n, 3)
    xt = torch.tensor(x, device="cuda:0")
    yt = torch.empty_like(xt)
    csrk.spmv(h, 1.0, xt, 0.0, yt)
    torch.cuda.synchronize()
    ref = ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x)
    s = ospmv.abs_row_scale(a.rowptr, a.colidx, a.vals, x)
    assert np.all(np.abs(yt.cpu().numpy() - ref) <= 1e-12 * s)
    assert csrk.device_status(h) == 0
    csrk.destroy(h)


# ------------------------------------------------------------------ host-side fault injection
def _mem_free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("step,status", [("alloc", "ERR_ALLOC"), ("h2d", "ERR_CUDA")])
def test_injected_upload_faults_fail_cleanly(step, status, monkeypatch):
    a = synth.stencil_3d(20, 20, 20, 7, "random_dd", 3)
    x = torch.tensor(synth.uniform_vector(a.n, 4), device="cuda:0")
    y = torch.empty_like(x)
    free0 = _mem_free()
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder(h)
    csrk.set_sizes(h, 32, 4)
    monkeypatch.setenv("CSRK_FAULT", step)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.spmv(h, 1.0, x, 0.0, y)
    assert ei.value.status == status
    monkeypatch.delenv("CSRK_FAULT")
    csrk.spmv(h, 1.0, x, 0.0, y)                     # the same handle works once the fault is gone
    torch.cuda.synchronize()
    ref = ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x.cpu().numpy())
    assert np.allclose(y.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    csrk.destroy(h)
    assert _mem_free() == free0                      # nothing leaked


def test_injected_tuning_and_solver_faults(monkeypatch):
    a = synth.stencil_3d(16, 16, 16, 27, "random_dd", 5)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder(h)
    monkeypatch.setenv("CSRK_FAULT", "tune")
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.set_sizes(h, 0, 0)
    assert ei.value.status == "ERR_CUDA"
    monkeypatch.setenv("CSRK_FAULT", "alloc")          # the CG workspace cannot be allocated
    csrk.set_sizes(h, 32, 4)
    b = torch.tensor(synth.uniform_vector(a.n, 6), device="cuda:0")
    xs = torch.zeros_like(b)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.cg(h, b, xs, 1e-10, 500, "f64")
    assert ei.value.status == "ERR_ALLOC"
    monkeypatch.delenv("CSRK_FAULT")
    csrk.set_sizes(h, 0, 0)
    rc, iters, rel = csrk.cg(h, b, xs, 1e-10, 500, "f64")
    assert rc == 0 and rel <= 1e-10
    csrk.destroy(h)
