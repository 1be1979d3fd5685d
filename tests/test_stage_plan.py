"""The TMA kernels' shared-memory stage layout (host only, no GPU): for every SSR the tile
statistics admit, each slice the producer copies -- rounded out to 16-byte boundaries at
both ends, from any starting element -- fits the region the plan gives it, the regions do
not overlap, and the stages plus their mbarrier/descriptor header fit the shared memory
the plan was made for.  A slice that overran its region would corrupt the next one while
its copy is in flight, so this is the staging's memory-safety contract."""
import numpy as np
import pytest

from paper_2203_05096_gb300 import csrk


def worst_slice(count, esz):
    """Largest byte count of a copy of `count` elements of `esz` bytes rounded out to
    16-byte boundaries at both ends, over every alignment of its first element."""
    per = 16 // esz
    best = 0
    for first in range(per):
        a0 = first & ~(per - 1)
        a1 = (first + count + per - 1) & ~(per - 1)
        best = max(best, (a1 - a0) * esz)
    return best


def check(max_srs, max_rows, max_nnz, val_bytes, col_bytes, max_smem, want, x_bytes, with_ord):
    try:
        p = csrk.stage_plan(max_srs, max_rows, max_nnz, val_bytes, col_bytes, max_smem, want, x_bytes, with_ord)
    except csrk.CsrkError as e:
        assert e.status == "ERR_UNSUPPORTED"
        return None
    offs = [p["off_srp"], p["off_rp"], p["off_col"], p["off_val"], p["off_x"], p["off_perm"], p["off_ord"],
            p["stage_bytes"]]
    assert all(o % 16 == 0 for o in offs) and offs == sorted(offs) and p["off_srp"] == 0
    assert p["stage_bytes"] % 128 == 0
    region = dict(zip(("srp", "rp", "col", "val", "x", "perm", "ord"), np.diff(offs)))
    assert worst_slice(max_srs + 1, 4) <= region["srp"]            # sr_ptr[s0 .. s1]
    assert worst_slice(max_rows + 1, 4) <= region["rp"]            # rowptr[r0 .. r1]
    assert worst_slice(max_nnz, col_bytes) <= region["col"]
    assert worst_slice(max_nnz, val_bytes) <= region["val"]
    assert x_bytes <= region["x"]
    if x_bytes > 0 or col_bytes == 2:                              # the fused unpermute's slice
        assert worst_slice(max_rows, 4) <= region["perm"]
    if x_bytes > 0 and with_ord:
        assert worst_slice(max_rows, 2) <= region["ord"]
    s = p["stages"]
    assert 2 <= s <= 16 and (want == 0 or s <= want)
    assert p["header_bytes"] >= 48 * s and p["header_bytes"] % 16 == 0   # 2 mbarriers + a descriptor each
    assert s * p["stage_bytes"] + p["header_bytes"] <= max_smem
    return p


def test_stage_plan_random_tiles():
    rng = np.random.default_rng(2203)
    planned = 0
    for _ in range(3000):
        x_bytes = int(rng.choice([0, 0, 16 * int(rng.integers(1, 1025))]))
        p = check(int(rng.integers(1, 33)), int(rng.integers(1, 513)), int(rng.integers(0, 8001)),
                  int(rng.choice([2, 4, 8])), int(rng.choice([2, 4])),
                  int(rng.choice([48 * 1024, 75 * 1024, 113 * 1024, 232448])), int(rng.choice([0, 2, 3, 5, 16])),
                  x_bytes, bool(rng.integers(0, 2)))
        planned += p is not None
    assert planned > 1000


SM = 233472   # shared memory per SM on GB300; a block of b per SM gets SM // b - 1024 bytes


@pytest.mark.parametrize("args", [
    (2, 64, 1728, 8, 2, SM // 3 - 1024, 0, 8 * 752, False),     # 27-point 128^3 SSR of 64 rows, kernel 5
    (8, 256, 1792, 8, 2, SM // 4 - 1024, 0, 8 * 1044, False),   # 7-point SSR of 256 rows, 4 blocks per SM
    (4, 128, 2432, 8, 2, SM // 2 - 1024, 0, 8 * 2360, True),    # FEM-like SSR of 128 rows, length order
    (4, 128, 3456, 8, 4, SM // 2 - 1024, 0, 0, False),          # kernel 0
    (1, 1, 0, 8, 4, 49152, 0, 0, False),                            # an SSR of one empty row
])
def test_stage_plan_benchmark_shapes(args):
    assert check(*args) is not None


def test_stage_plan_refuses_what_does_not_fit_and_bad_arguments():
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.stage_plan(8, 256, 200000, 8, 4, 232448, 0)             # 2.4 MB of values a stage
    assert ei.value.status == "ERR_UNSUPPORTED"
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.stage_plan(8, 256, 1000, 3, 4, 232448, 0)
    assert ei.value.status == "ERR_ARG"
