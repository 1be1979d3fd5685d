"""Host side of the x-window kernels (5 and 6), no GPU: the windows, their 16-bit codes and the
rows' length order that the library builds (csrk_xwin_export) equal a separate numpy
construction from their definitions, and satisfy the properties the kernels rely on.

Definitions restated here: an SSR's window is the list of runs of aligned 4-element blocks
of x holding its columns, runs whose gap is at most 2 blocks merged; the runs sit one after
another in the window; a nonzero's code is its column's offset in the window; the window
is usable when every SSR's (block-aligned) window holds at most 65,536 elements.  The
length order hands an SSR's rows to the warp passes (32 positions of a super-row at a time)
by decreasing row length, ties in row order.
"""
import numpy as np
import pytest

import synth
from paper_2203_05096_gb300 import csrk

ALIGN, GAP, LIMIT = 4, 2, 65536


def ssr_ranges(e):
    srp, ssrp, rp = e["sr_ptr"], e["ssr_ptr"], e["rowptr"]
    for t in range(len(ssrp) - 1):
        r0, r1 = int(srp[ssrp[t]]), int(srp[ssrp[t + 1]])
        yield t, int(ssrp[t]), int(ssrp[t + 1]), r0, r1, int(rp[r0]), int(rp[r1])


def expected_windows(n, e):
    """Per SSR: the runs as (start, base) pairs, the covered element count and the aligned
    window length, and the code of every nonzero."""
    codes = np.zeros(len(e["colidx"]), np.int64)
    out = []
    for t, _, _, _, _, p0, p1 in ssr_ranges(e):
        cols = e["colidx"][p0:p1].astype(np.int64)
        blocks = np.unique(cols // ALIGN)
        runs, base, cover = [], 0, 0
        i = 0
        while i < len(blocks):
            first = last = int(blocks[i])
            while i + 1 < len(blocks) and blocks[i + 1] - last <= GAP + 1:
                i += 1
                last = int(blocks[i])
            i += 1
            start, end = first * ALIGN, min((last + 1) * ALIGN, n)
            runs.append((start, base))
            cover = base + (end - start)
            base += (last - first + 1) * ALIGN
        starts = np.array([r[0] for r in runs], np.int64)
        bases = np.array([r[1] for r in runs], np.int64)
        k = np.searchsorted(starts, cols, side="right") - 1
        codes[p0:p1] = bases[k] + cols - starts[k]
        out.append((runs, cover, base))
    return out, codes


def expected_order(e):
    rp, srp = e["rowptr"], e["sr_ptr"]
    length = np.diff(rp)
    covered = int(srp[-1]) if len(srp) else 0
    ord_ = np.zeros(covered, np.int64)
    nat = srt = 0
    for _, s0, s1, r0, r1, _, _ in ssr_ranges(e):
        rows = r0 + np.argsort(-length[r0:r1], kind="stable")
        ord_[r0:r1] = rows - r0
        for sr in range(s0, s1):
            for q in range(int(srp[sr]), int(srp[sr + 1]), 32):
                q1 = min(q + 32, int(srp[sr + 1]))
                nat += int(length[q:q1].max())
                srt += int(length[rows[q - r0:q1 - r0]].max())
    return ord_, (nat, srt)


def check(a, sr, ssr, reorder=True, split=0):
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    if reorder:
        csrk.reorder(h)
    if split:
        csrk.split_long_rows(h, split)
    csrk.set_sizes(h, sr, ssr)
    e = csrk.export(h)
    got = csrk.xwin_export(h)
    wins, codes = expected_windows(a.n, e)
    ok = all(w[2] <= LIMIT for w in wins)
    assert got["available"] == ok
    if ok:
        runs = [r for w in wins for r in w[0]]
        assert np.array_equal(got["win"], np.array(runs, np.int32).reshape(-1, 2))
        assert np.array_equal(np.diff(got["wptr"]), [len(w[0]) for w in wins]) and got["wptr"][0] == 0
        assert np.array_equal(got["cover"], [w[1] for w in wins])
        assert np.array_equal(got["codes"].astype(np.int64), codes)
        # what the kernels rely on: every code decodes to its column, runs are aligned and
        # inside x, the window fits the 16-bit offsets
        for t, _, _, _, _, p0, p1 in ssr_ranges(e):
            w = got["win"][got["wptr"][t]:got["wptr"][t + 1]].astype(np.int64)
            assert np.all(w[:, 0] % ALIGN == 0) and np.all(w[:, 1] % ALIGN == 0)
            assert np.all(np.diff(w[:, 0]) > 0) and np.all(np.diff(w[:, 1]) > 0)
            c = got["codes"][p0:p1].astype(np.int64)
            k = np.searchsorted(w[:, 1], c, side="right") - 1
            assert np.array_equal(w[k, 0] + c - w[k, 1], e["colidx"][p0:p1])
            assert np.all(c < got["cover"][t]) and got["cover"][t] <= LIMIT
            assert w[-1, 0] + got["cover"][t] - w[-1, 1] <= a.n
    ord_, slots = expected_order(e)
    assert np.array_equal(got["ord"].astype(np.int64), ord_)
    assert got["slots"] == slots and slots[1] <= slots[0]
    csrk.destroy(h)
    return got, e


@pytest.mark.parametrize("sizes", [(32, 1), (32, 4), (16, 8), (64, 2)])
def test_windows_stencils(sizes):
    for a in (synth.stencil_3d(12, 11, 10, 7, "random_dd", 1, labels=synth.vectors.permutation(1320, 1)),
              synth.stencil_3d(9, 10, 11, 27, "random_dd", 2, labels=synth.vectors.permutation(990, 2))):
        got, _ = check(a, *sizes)
        assert got["available"]


@pytest.mark.parametrize("sizes", [(32, 2), (32, 4)])
def test_windows_fem_like_and_row_order(sizes):
    """Rows of 13-24 entries: the length order saves FP64 slots on every SSR size."""
    got, _ = check(synth.fem_like(9, 3), *sizes)
    nat, srt = got["slots"]
    assert srt < nat


def test_windows_random_patterns_empty_rows_and_no_reorder():
    check(synth.random_pattern(3000, 0.003, 11, empty_rows=80), 32, 4)
    check(synth.random_pattern(2500, 0.004, 12, empty_rows=40), 32, 2, reorder=False)


def test_windows_too_wide_are_refused():
    """Without reordering, a scrambled 7-point grid's 4,096-row SSRs have windows over 65,536 elements:
    the windows are reported unavailable (and the row order is still built)."""
    a = synth.stencil_3d(50, 50, 50, 7, "random_dd", 5, labels=synth.vectors.permutation(50 ** 3, 5))
    got, _ = check(a, 64, 64, reorder=False)
    assert not got["available"]


def test_windows_skip_split_long_rows():
    """Rows split off as long rows are in no SSR: their entries carry code 0, and the
    length order covers the other rows only."""
    a = synth.with_dense_rows(synth.stencil_3d(10, 10, 10, 7, "random_dd", 6), 3, 700, 7)
    got, e = check(a, 32, 4, split=512)
    assert got["available"] and len(got["ord"]) == a.n - 3
    assert not got["codes"][e["rowptr"][a.n - 3]:].any()
