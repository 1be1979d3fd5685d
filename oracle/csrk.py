"""Oracle CSR-k pointer arrays (TEST INFRASTRUCTURE).

Sec. 2.2 and Fig. 1: CSR-3 adds ``sr_ptr`` (running count of rows, one entry per
super-row plus a leading 0) and ``ssr_ptr`` (running count of super-rows, one entry per
super-super-row plus a leading 0), compressed the way ``row_ptr`` compresses nonzeros.
A super-row is a run of contiguous rows, a super-super-row a run of contiguous
super-rows.  Fig. 1's example: sr_ptr = {0,2,5,7,9}, ssr_ptr = {0,2,4}; the number of
super-super-rows is len(ssr_ptr) - 1 (the text's "num_ssr = 3" for that figure disagrees
with its own array; the array is taken as authoritative).

Fixed sizes (the library's ``csrk_set_sizes(sr, ssr)``): every super-row holds ``sr`` rows
and every super-super-row ``ssr`` super-rows, the last of each possibly fewer.

Pins (tests/test_oracle_csrk.py): hand-worked pointer arrays in
tests/golden/csrk_pointers.txt; Fig. 1's arrays drive the Listing 1 loop nest to the
plain CSR result; structural invariants (first 0, last n / nsr, non-decreasing, group
sizes) checked by a separate validator.
"""
from __future__ import annotations

import numpy as np


def fixed_pointers(n: int, sr: int, ssr: int):
    """(sr_ptr, ssr_ptr) for fixed group sizes, built by walking rows and super-rows."""
    if sr <= 0 or ssr <= 0:
        raise ValueError("sizes must be positive")
    sr_ptr = [0]
    rows_left = n
    while rows_left > 0:
        take = min(sr, rows_left)
        sr_ptr.append(sr_ptr[-1] + take)
        rows_left -= take
    nsr = len(sr_ptr) - 1
    ssr_ptr = [0]
    srs_left = nsr
    while srs_left > 0:
        take = min(ssr, srs_left)
        ssr_ptr.append(ssr_ptr[-1] + take)
        srs_left -= take
    return np.array(sr_ptr, dtype=np.int32), np.array(ssr_ptr, dtype=np.int32)


def validate_pointers(n: int, sr_ptr, ssr_ptr):
    """Structural rules of Sec. 2.2; returns a list of violations."""
    errs = []
    sr_ptr = np.asarray(sr_ptr, dtype=np.int64)
    ssr_ptr = np.asarray(ssr_ptr, dtype=np.int64)
    if sr_ptr.size < 1 or sr_ptr[0] != 0 or sr_ptr[-1] != n:
        errs.append("sr_ptr must start at 0 and end at n")
    if np.any(np.diff(sr_ptr) < 0):
        errs.append("sr_ptr decreases")
    nsr = sr_ptr.size - 1
    if ssr_ptr.size < 1 or ssr_ptr[0] != 0 or ssr_ptr[-1] != nsr:
        errs.append("ssr_ptr must start at 0 and end at the number of super-rows")
    if np.any(np.diff(ssr_ptr) < 0):
        errs.append("ssr_ptr decreases")
    return errs
