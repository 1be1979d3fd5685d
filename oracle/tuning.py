"""Oracle of the paper's constant-time super-row size model (TEST INFRASTRUCTURE).

Sec. 4.1: with rdensity = NNZ / N, the super-super-row size SSRS and super-row size SRS
come from a logarithmic fit, rounded to nearest with halves toward +infinity
(round(v) = floor(v + 1/2)):

    Volta:  SSRS = round(8.900 - 1.25 ln r),  SRS = round(10.146 - 1.50 ln r)
    Ampere: SSRS = round(9.175 - 1.32 ln r),  SRS = round(20.500 - 3.50 ln r)

then adjusted by the rdensity case (case 1: r <= 8, case 2: 8 < r <= 16,
case 3: 16 < r <= 32, case 4: r > 32):

    Volta:  c2: SSRS = round(1.5 SSRS), SRS = 2 SRS;  c3: SSRS = 4 SSRS, SRS = floor(SSRS/2);
            c4: SSRS = 5 SSRS, SRS = floor(SSRS/2)
    Ampere: c2: SRS = 4 SRS;  c3: SSRS = round(2.5 SSRS), SRS = 3 SSRS;
            c4: SSRS = 2 SSRS, SRS = 2 SSRS

Readings: "SRSS" in the case tables is a typo for SRS; each case's two assignments run
top to bottom, so the SRS rule sees the SSRS just updated.  The same section fixes the
GPU block shapes per case (x*y*z threads): 8x12, 4x8x12, 8x8x8, 16x8x4, and the tuning
search grid {2^i, 1.5*2^i : i = 2..5} for both sizes.

Pins (tests/test_oracle_tuning.py): values worked by hand in tests/golden/tuning_model.txt.
"""
from __future__ import annotations

import math

COEFFS = {"volta": (8.900, 1.25, 10.146, 1.50), "ampere": (9.175, 1.32, 20.500, 3.50)}
BLOCK_DIMS = {1: (8, 12, 1), 2: (4, 8, 12), 3: (8, 8, 8), 4: (16, 8, 4)}


def round_half_up(v: float) -> int:
    return math.floor(v + 0.5)


def case_of(rdensity: float) -> int:
    if rdensity <= 8:
        return 1
    if rdensity <= 16:
        return 2
    if rdensity <= 32:
        return 3
    return 4


def model_sizes(rdensity: float, arch: str = "ampere"):
    """(SSRS, SRS) of the paper's model for a GPU generation ("volta" or "ampere")."""
    a, b, c, d = COEFFS[arch]
    lr = math.log(rdensity)
    ssrs = round_half_up(a - b * lr)
    srs = round_half_up(c - d * lr)
    case = case_of(rdensity)
    if arch == "volta":
        if case == 2:
            ssrs = round_half_up(ssrs * 1.5)
            srs = srs * 2
        elif case == 3:
            ssrs = ssrs * 4
            srs = ssrs // 2
        elif case == 4:
            ssrs = ssrs * 5
            srs = ssrs // 2
    else:
        if case == 2:
            srs = srs * 4
        elif case == 3:
            ssrs = round_half_up(ssrs * 2.5)
            srs = ssrs * 3
        elif case == 4:
            ssrs = ssrs * 2
            srs = ssrs * 2
    return ssrs, srs


def search_grid():
    """{2^i, 1.5*2^i : i = 2..5}, the candidate sizes of Sec. 4.1."""
    out = set()
    for i in range(2, 6):
        out.add(2 ** i)
        out.add(int(1.5 * 2 ** i))
    return sorted(out)
