"""The FP32-integrate kernels' own precision conversions, bit for bit against
IEEE 754 (numpy's conversions): FP32 -> FP64 widening, which every FP32
element contribution takes into the FP64 accumulation, and FP64 -> FP32
round-to-nearest-even, which the FP64 geometry takes into the FP32 records.
Both are integer-instruction code paths (the FP64 pipe is kept for the
arithmetic), so every class of input is covered: zeros, subnormals, the
normal range's ends, infinities, NaNs, and random bit patterns."""
import numpy as np
import pytest

from tests.helpers import engine

pytestmark = pytest.mark.gpu


def _bits32(rng, n):
    special = np.array([0x00000000, 0x80000000, 0x00000001, 0x80000001, 0x007fffff, 0x807fffff, 0x00800000,
                        0x80800000, 0x7f7fffff, 0xff7fffff, 0x3f800000, 0xbf800000, 0x7f800000, 0xff800000,
                        0x7fc00000, 0xffc00001, 0x7f800001, 0x00400000, 0x33800000], dtype=np.uint32)
    rnd = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    sub = rng.integers(0, 0x00800000, size=n // 8, dtype=np.uint32) | (rng.integers(0, 2, size=n // 8,
                                                                                   dtype=np.uint32) << 31)
    return np.concatenate([special, rnd, sub])


def test_widening_is_exact():
    import torch
    fea = engine()
    u = _bits32(np.random.default_rng(11), 1 << 20)
    x = u.view(np.float32)
    got = fea.fea_convert(torch.from_numpy(x.copy()).cuda()).cpu().numpy()
    with np.errstate(invalid="ignore"):
        want = x.astype(np.float64)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint64), want[~nan].view(np.uint64))


def test_rounding_is_nearest_even():
    import torch
    fea = engine()
    rng = np.random.default_rng(12)
    n = 1 << 20
    # random patterns, values near the FP32 range ends and subnormals, exact
    # ties (a 1 just below the kept bits, half-way) and one above / below them
    rnd = rng.integers(0, 2**64, size=n, dtype=np.uint64)
    mid = rng.uniform(-1e3, 1e3, size=n).astype(np.float32).astype(np.float64).view(np.uint64)
    tie = mid | np.uint64(1 << 28)
    near = np.concatenate([tie, tie + np.uint64(1), tie - np.uint64(1)])
    ends = np.array([3.4028234663852886e38, 3.4028235677973366e38, 3.4028236e38, 1.1754943508222875e-38,
                     1.1754942e-38, 1.401298464324817e-45, 7.006492321624085e-46, 7.0e-46, 1e-50, 0.0, -0.0,
                     np.inf, -np.inf, np.nan, 1.0 + 2.0**-24, 1.0 + 3 * 2.0**-24, 1.0 - 2.0**-25],
                    dtype=np.float64).view(np.uint64)
    # results in the binary32 subnormal range: every multiple of 2^-150 up to
    # 2^-138 (the odd ones are exact ties between neighbouring subnormals) and
    # the doubles just above and below them, and random doubles there
    k = np.ldexp(np.arange(-4096, 4097, dtype=np.float64), -150)
    sub = np.concatenate([k, np.nextafter(k, np.inf), np.nextafter(k, -np.inf),
                          np.ldexp(rng.uniform(-1.0, 1.0, size=4096), -126 - rng.integers(0, 26, size=4096))])
    b = np.concatenate([rnd, near, ends, sub.view(np.uint64)])
    x = b.view(np.float64)
    got = fea.fea_convert(torch.from_numpy(x.copy()).cuda()).cpu().numpy()
    with np.errstate(over="ignore", invalid="ignore"):
        want = x.astype(np.float32)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint32), want[~nan].view(np.uint32))


def test_empty_and_bad_arguments():
    import torch
    fea = engine()
    assert fea.fea_convert(torch.empty(0, dtype=torch.float32, device="cuda")).numel() == 0
    with pytest.raises(TypeError):
        fea.fea_convert(torch.zeros(4, dtype=torch.float16, device="cuda"))
