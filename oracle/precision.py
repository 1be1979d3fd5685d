"""Oracle precision conversion (TEST INFRASTRUCTURE).

The stored values of A may be narrowed from FP64 to FP32 or BF16 (the library's value
dtypes; the paper's own storage examples assume 32-bit values, Sec. 2.1).  Rounding is
IEEE round-to-nearest, ties to even, applied once, directly from the FP64 value (never
through FP32 first, which can round twice).  NaN stays NaN (quiet), values beyond the
largest finite BF16 after rounding become +-Inf, and BF16 subnormals are kept.

BF16: 1 sign bit, 8 exponent bits (bias 127, as FP32), 7 stored fraction bits, so
8 significant bits for normal numbers; the smallest normal is 2^-126 and the subnormal
quantum 2^-133.

Pins (tests/test_oracle_precision.py): FP32 equals the C cast (numpy astype, IEEE RNE);
on FP32-representable inputs BF16 equals torch's float32 -> bfloat16 conversion;
hand-worked halfway, double-rounding, overflow, subnormal and NaN cases in
tests/golden/bf16_cases.txt.
"""
from __future__ import annotations

import math
import struct

import numpy as np


def to_f32(vals) -> np.ndarray:
    """FP64 -> FP32, IEEE round-to-nearest-even (numpy's cast)."""
    return np.asarray(vals, dtype=np.float64).astype(np.float32)


def _bf16_of(d: float) -> int:
    """Bit pattern of the BF16 nearest to the double d (ties to even)."""
    if math.isnan(d):
        return 0x7FC0 | (0x8000 if math.copysign(1.0, d) < 0 else 0)
    sign = 0x8000 if math.copysign(1.0, d) < 0 else 0
    a = abs(d)
    if a == 0.0:
        return sign
    if math.isinf(a):
        return sign | 0x7F80
    _, e = math.frexp(a)          # a = m * 2**e, 0.5 <= m < 1, so a in [2**(e-1), 2**e)
    exp = e - 1                   # a in [2**exp, 2**(exp+1))
    q_exp = max(exp, -126) - 7    # spacing of BF16 values around a
    scaled = math.ldexp(a, -q_exp)    # exact: a power-of-two scaling of a double
    m = round(scaled)             # Python rounds exact halves to even
    value = math.ldexp(m, q_exp)
    if value > math.ldexp(255.0, 120):   # largest finite BF16 = (2 - 2**-7) * 2**127
        return sign | 0x7F80
    bits32 = struct.unpack("<I", struct.pack("<f", value))[0]   # value is a BF16, so exact
    return sign | (bits32 >> 16)


def to_bf16_bits(vals) -> np.ndarray:
    """FP64 -> BF16 bit patterns (uint16), one value at a time."""
    flat = np.asarray(vals, dtype=np.float64).reshape(-1)
    return np.array([_bf16_of(float(v)) for v in flat], dtype=np.uint16)


def bf16_bits_to_f64(bits) -> np.ndarray:
    """Widen BF16 bit patterns to FP64 (exact)."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)
