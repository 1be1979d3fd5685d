"""Pins of the FP64 -> FP32 / BF16 rounding oracle."""
import math

import numpy as np
import torch

from oracle import precision
from tests.conftest import read_golden


def test_hand_worked_bf16_cases():
    for expr, hexbits, why in read_golden("bf16_cases.txt"):
        v = eval(expr, {"float": float})
        got = int(precision.to_bf16_bits([v])[0])
        assert got == int(hexbits, 16), f"{expr}: {got:04X} != {hexbits} ({why})"


def test_bf16_matches_torch_on_fp32_inputs():
    rng = np.random.default_rng(3)
    f = np.concatenate([rng.standard_normal(4000).astype(np.float32),
                        (rng.standard_normal(2000) * 1e-38).astype(np.float32),
                        (rng.standard_normal(2000) * 1e37).astype(np.float32),
                        rng.integers(0, 2**32, size=4000, dtype=np.uint64).astype(np.uint32).view(np.float32)])
    f = f[np.isfinite(f)]
    ref = torch.from_numpy(f).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = precision.to_bf16_bits(f.astype(np.float64))
    assert np.array_equal(got, ref)


def test_f32_is_ieee_cast():
    vals = [1 + 2**-24, 1 + 3 * 2**-24, 1e-45, 3.4028235677973366e38, 1e39, -0.0]
    got = precision.to_f32(vals)
    assert got[0] == np.float32(1.0)                 # tie to even
    assert got[1] == np.float32(1 + 2**-22)          # tie to even, upward
    assert got[2] == np.float32(1.401298464324817e-45)
    assert np.isinf(got[4])
    assert math.copysign(1.0, float(got[5])) < 0


def test_widen_roundtrip():
    bits = np.arange(0, 65536, 7, dtype=np.uint16)
    w = precision.bf16_bits_to_f64(bits)
    fin = np.isfinite(w)
    back = precision.to_bf16_bits(w[fin])
    assert np.array_equal(back, bits[fin])
