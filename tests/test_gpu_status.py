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
