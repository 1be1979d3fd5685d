"""The solvers' FP64 -> FP32 narrowing (integer round to nearest, ties to even; used for
the FP32 copies of p in the mixed-precision CG and the batched solver) against two
independent references: numpy's IEEE conversion on the host and the GPU's conversion
instruction, bit for bit, on random bit patterns over every exponent, on exact and near
ties at the rounding cut (normal and subnormal FP32 results), and on the range edges."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05096_gb300 import csrk  # noqa: E402

DEV = "cuda:0"


def _inputs(n=1 << 22, seed=17):
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2 ** 63, n, dtype=np.int64).view(np.uint64) | (
        rng.integers(0, 2, n).astype(np.uint64) << np.uint64(63))
    sign = bits & np.uint64(1 << 63)
    q = n // 4
    # exponents around the FP32 range (FP32 overflow, normal, subnormal, underflow)
    e = rng.integers(1023 - 160, 1023 + 140, q).astype(np.uint64)
    bits[q:2 * q] = sign[q:2 * q] | (e << np.uint64(52)) | (bits[q:2 * q] & np.uint64((1 << 52) - 1))
    # ties and near ties at the 29-bit cut of a normal FP32 result
    e = rng.integers(1023 - 120, 1023 + 120, q).astype(np.uint64)
    m = rng.integers(0, 1 << 52, q, dtype=np.int64).astype(np.uint64) & ~np.uint64((1 << 29) - 1)
    k = rng.integers(0, 4, q)
    low = np.where(k == 0, 1 << 28, np.where(k == 1, (1 << 28) - 1, np.where(k == 2, (1 << 28) + 1, 0)))
    bits[2 * q:3 * q] = sign[2 * q:3 * q] | (e << np.uint64(52)) | m | low.astype(np.uint64)
    # FP32 subnormal results, half of them exact ties
    e = rng.integers(1023 - 155, 1023 - 126, q)
    m = rng.integers(0, 1 << 52, q, dtype=np.int64).astype(np.uint64)
    drop = 30 + (1023 - 127 - e)                 # bits below the FP32 subnormal unit
    tie = rng.integers(0, 2, q).astype(bool) & (drop < 53)
    dm = np.minimum(drop, 52).astype(np.uint64)
    m = np.where(tie, (m & ~((np.uint64(1) << dm) - np.uint64(1))) | (np.uint64(1) << (dm - np.uint64(1))), m)
    bits[3 * q:] = sign[3 * q:] | (e.astype(np.uint64) << np.uint64(52)) | (m & np.uint64((1 << 52) - 1))
    x = bits.view(np.float64).copy()
    x[np.isnan(x)] = 1.5                          # NaNs have their own test
    f32max = float(np.finfo(np.float32).max)
    edges = [0.0, -0.0, 1.0, -1.0, f32max, -f32max, np.nextafter(f32max, np.inf),
             f32max * (1 + 2.0 ** -25), f32max * (1 + 2.0 ** -24), 1e39, -1e39,
             float(np.finfo(np.float32).tiny), float(np.finfo(np.float32).smallest_subnormal),
             float(np.finfo(np.float32).smallest_subnormal) / 2,
             np.nextafter(float(np.finfo(np.float32).smallest_subnormal) / 2, 1.0),
             5e-324, 1e-300, np.inf, -np.inf]
    x[:len(edges)] = edges
    return x


def test_integer_narrowing_matches_ieee_and_the_conversion_instruction():
    x = _inputs()
    xt = torch.tensor(x, device=DEV)
    by_int = torch.empty(x.size, dtype=torch.float32, device=DEV)
    by_cvt = torch.empty_like(by_int)
    csrk.selftest_narrow(xt, by_int, by_cvt)
    torch.cuda.synchronize()
    a = by_int.cpu().numpy().view(np.uint32)
    c = by_cvt.cpu().numpy().view(np.uint32)
    with np.errstate(over="ignore"):
        h = x.astype(np.float32).view(np.uint32)
    nan = np.isnan(x)
    assert not nan.any()
    assert np.array_equal(a, h), f"{np.count_nonzero(a != h)} differ from numpy"
    assert np.array_equal(a, c), f"{np.count_nonzero(a != c)} differ from the instruction"
    # the draw reaches every regime it is meant to
    f = by_int.cpu().numpy()
    assert np.isinf(f).any() and (f == 0).any() and (np.abs(f[f != 0]) < np.finfo(np.float32).tiny).any()


def test_integer_narrowing_nan_stays_nan():
    x = np.array([np.nan, -np.nan, np.frombuffer(np.uint64(0x7FF0000000000001).tobytes(), np.float64)[0]])
    xt = torch.tensor(x, device=DEV)
    by_int = torch.empty(3, dtype=torch.float32, device=DEV)
    by_cvt = torch.empty_like(by_int)
    csrk.selftest_narrow(xt, by_int, by_cvt)
    torch.cuda.synchronize()
    assert torch.isnan(by_int).all() and torch.isnan(by_cvt).all()
