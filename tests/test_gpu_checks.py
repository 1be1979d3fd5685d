"""The bounds-checked build (libcsrk_checks.so, CSRK_CHECKS=1): on valid inputs its checks
never fire and its results equal the regular build's bit for bit.

The checked build stands in for a memory checker on this GPU pool: every CSR-3 kernel
checks each index it is about to follow (row and nonzero ranges, columns, window
offsets, unpermute targets) and skips, with status bit 1 set, anything out of bounds.
A child process loads the checked library (the binding picks it from the environment),
runs every SpMV kernel, an SpMM and a matrix with split long rows, and saves the results;
this process runs the same calls on the regular library and compares.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05096_gb300 import csrk  # noqa: E402
from tests.conftest import ROOT  # noqa: E402

DEV = "cuda:0"
CASES = [dict(kernel=0, lanes=1, unroll=8), dict(kernel=1, lanes=1, unroll=8), dict(kernel=0, lanes=4, unroll=8),
         dict(kernel=4, lanes=1, unroll=8), dict(kernel=5, lanes=1, unroll=4, warps=8),
         dict(kernel=6, lanes=1, unroll=8, warps=8), dict(kernel=2, lanes=1, unroll=8)]


def run_cases(out_path):
    """Every case's y (and status word) on the library this process loaded."""
    res = {}
    a = synth.stencil_3d(20, 17, 15, 27, "random_dd", 51, labels=synth.vectors.permutation(5100, 51))
    x = torch.tensor(synth.uniform_vector(a.n, 52), device=DEV)
    y0 = torch.tensor(synth.uniform_vector(a.n, 53), device=DEV)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder(h)
    csrk.set_sizes(h, 32, 4)
    for i, cfg in enumerate(CASES):
        csrk.set_config(h, **cfg)
        y = y0.clone()
        csrk.spmv(h, 1.5, x, -0.5, y)
        torch.cuda.synchronize()
        res[f"spmv{i}"] = y.cpu().numpy()
        res[f"status{i}"] = np.array([csrk.device_status(h)])
    X = torch.tensor(synth.uniform_block(a.n, 3, 54), device=DEV)
    Y = torch.empty_like(X)
    csrk.set_config(h, kernel=0, lanes=1, unroll=8)
    csrk.spmm(h, 3, 1.0, X, 3, 0.0, Y, 3)
    torch.cuda.synchronize()
    res["spmm"] = Y.cpu().numpy()
    res["status_spmm"] = np.array([csrk.device_status(h)])
    csrk.destroy(h)
    b = synth.with_dense_rows(a, 3, 4500, 55)
    h = csrk.create(b.n, b.rowptr, b.colidx, b.vals)
    csrk.reorder(h)
    csrk.split_long_rows(h, 2048)
    csrk.set_sizes(h, 32, 4)
    csrk.set_config(h, kernel=5, lanes=1, unroll=8, warps=8)
    y = torch.empty_like(x)
    csrk.spmv(h, 1.0, x, 0.0, y)
    torch.cuda.synchronize()
    res["long"] = y.cpu().numpy()
    res["status_long"] = np.array([csrk.device_status(h)])
    csrk.destroy(h)
    res["build_info"] = np.array([csrk.lib().csrk_build_info().decode()])
    np.savez(out_path, **res)


def test_checked_build_agrees_and_stays_quiet(tmp_path):
    checked = tmp_path / "checked.npz"
    env = dict(os.environ, CSRK_CHECKS="1")
    code = ("import sys; sys.path.insert(0, {root!r}); from tests.test_gpu_checks import run_cases; "
            "run_cases({out!r})").format(root=ROOT, out=str(checked))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    regular = tmp_path / "regular.npz"
    run_cases(str(regular))
    c, g = np.load(checked), np.load(regular)
    assert "bounds checks on" in str(c["build_info"][0]) and "bounds checks" not in str(g["build_info"][0])
    for k in g.files:
        if k == "build_info":
            continue
        if k.startswith("status"):
            assert int(c[k][0]) == 0 and int(g[k][0]) == 0, (k, json.dumps([int(c[k][0]), int(g[k][0])]))
        else:
            assert np.array_equal(c[k], g[k]), k
