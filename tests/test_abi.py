"""The C-ABI library loads, exports every symbol its header declares, and rejects bad
input on the host (no GPU needed)."""
import re

import numpy as np
import pytest

import synth
from paper_2203_05096_gb300 import csrk
from tests.conftest import ROOT


def declared_symbols():
    import os
    out = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            text = open(os.path.join(ROOT, "include", name)).read()
            out |= set(re.findall(r"^\s*(?:int|const char\*|void)\s+(csrk_\w+)\s*\(", text, re.M))
    return out


def test_library_exports_every_declared_symbol():
    lib = csrk.lib()
    syms = declared_symbols()
    assert "csrk_spmv" in syms and "csrk_create" in syms
    for s in sorted(syms):
        assert hasattr(lib, s), s


def _csr(rowptr, colidx, vals=None):
    rowptr = np.array(rowptr, np.int32)
    colidx = np.array(colidx, np.int32)
    vals = np.ones(colidx.size) if vals is None else np.array(vals, np.float64)
    return rowptr.size - 1, rowptr, colidx, vals


@pytest.mark.parametrize("bad,code", [
    (([1, 2, 3], [0, 1]), 2),                 # rowptr[0] != 0
    (([0, 2, 1], [0, 1]), 2),                 # decreasing rowptr
    (([0, 1, 2], [0, 2]), 2),                 # column out of range
    (([0, 2, 3], [1, 1, 0]), 2),              # repeated column
    (([0, 1, 2], [0, -1]), 2),                # negative column
])
def test_invalid_csr_rejected(bad, code):
    n, rp, ci, v = _csr(*bad)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.create(n, rp, ci, v)
    assert ei.value.code == code


def test_unsorted_rows_are_sorted_with_values():
    n, rp, ci, v = _csr([0, 3, 4, 6], [2, 0, 1, 1, 2, 0], [3.0, 1.0, 2.0, 4.0, 6.0, 5.0])
    h = csrk.create(n, rp, ci, v)
    e = csrk.export(h, with_pointers=False)
    assert e["colidx"].tolist() == [0, 1, 2, 1, 0, 2]
    assert e["vals"].tolist() == [1.0, 2.0, 3.0, 4.0, 5.0, 6.0]
    csrk.destroy(h)


def test_life_cycle_errors():
    a = synth.stencil_2d_5pt(4, 4)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.spmv(h, 1.0, 1, 0.0, 2)              # before the pointers exist
    assert ei.value.status == "ERR_STATE"
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.set_sizes(h, -1, 4)
    assert ei.value.status == "ERR_ARG"
    csrk.set_sizes(h, 4, 2)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.reorder(h)
    assert ei.value.status == "ERR_STATE"
    with pytest.raises(csrk.CsrkError):
        csrk.set_pointers(h, [0, 5, 16], [0, 1])   # ssr_ptr must end at nsr = 2
    with pytest.raises(csrk.CsrkError):
        csrk.set_pointers(h, [0, 5, 15], [0, 2])   # sr_ptr must end at n
    csrk.set_pointers(h, [0, 5, 16], [0, 2])
    assert csrk.info(h)["nsr"] == 2 and csrk.info(h)["sr"] == 0
    with pytest.raises(csrk.CsrkError):
        csrk.set_config(h, lanes=3)
    with pytest.raises(csrk.CsrkError):
        csrk.set_config(h, warps=17)
    csrk.destroy(h)
    csrk.destroy(None)


def test_unsupported_precision_combination_reported_before_gpu():
    a = synth.stencil_2d_5pt(4, 4)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, "f64")
    csrk.set_sizes(h, 4, 2)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.spmv(h, 1.0, 1, 0.0, 2, flags=csrk.X_F32)
    assert ei.value.status == "ERR_UNSUPPORTED"
    csrk.destroy(h)


def test_empty_matrix_host_side():
    h = csrk.create(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert csrk.reorder(h).size == 0
    csrk.set_sizes(h, 32, 8)
    assert csrk.info(h)["nsr"] == 0 and csrk.info(h)["nssr"] == 0
    csrk.destroy(h)


def test_selftest_narrow_arguments_checked_on_the_host():
    lib = csrk.lib()
    assert lib.csrk_selftest_narrow(None, -1, None, None, None) == 1     # CSRK_ERR_ARG
    assert lib.csrk_selftest_narrow(None, 5, None, None, None) == 1      # NULL arrays for n > 0
    assert lib.csrk_selftest_narrow(None, 0, None, None, None) == 0      # nothing to do, no launch
