"""The FP32 <-> FP64 conversions the mixed-precision recovery does on bit
patterns (widening of its FP32 operands, rounding of the FP64 pressure to
FP32), checked against IEEE-754 conversions by numpy (round to nearest, ties
to even) on random values, exact ties, overflow, infinities, NaNs and the
flushed subnormal range; on the GPU against the conversion instructions and
against the host evaluation of the same routines."""
import numpy as np
import pytest

from paper_1110_1616_gb300 import amrmhd

TINY = 2.0 ** -126  # smallest FP32 normal


def _doubles(seed, n=200000):
    rng = np.random.default_rng(seed)
    mag = np.exp2(rng.uniform(-140.0, 130.0, n))
    x = mag * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    # exact midpoints between neighbouring FP32 values (ties), even and odd
    f = rng.uniform(-1e6, 1e6, n // 4).astype(np.float32)
    g = np.nextafter(f, np.float32(np.inf))
    ties = (f.astype(np.float64) + g.astype(np.float64)) / 2.0
    fmax = float(np.finfo(np.float32).max)
    ulp = fmax - float(np.nextafter(np.float32(fmax), np.float32(0)))
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, fmax + ulp / 2, fmax + ulp / 4,
                        2.0 ** 128, TINY, -TINY, TINY / 3, 1e-300, 5e-324, 1.0, 2.0 / 3.0, 1.0 + 2.0 ** -24,
                        1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -24 + 2.0 ** -52])
    return np.concatenate([x, ties, special])


def _floats(seed, n=200000):
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -2.5, 1e-45, -1e-40, TINY,
                        float(np.finfo(np.float32).max)], dtype=np.float32)
    return np.concatenate([bits.view(np.float32), special])


def _expect_narrow(x):
    with np.errstate(over="ignore", invalid="ignore"):
        e = x.astype(np.float32)
    small = np.abs(x) < TINY
    e[small] = np.copysign(np.float32(0), x[small]).astype(np.float32)
    return e


def _expect_widen(y):
    with np.errstate(invalid="ignore"):
        e = y.astype(np.float64)
    sub = (y.view(np.uint32) & 0x7F800000) == 0
    e[sub] = np.copysign(0.0, y[sub].astype(np.float64))
    return e


def _same_bits(a, b):
    """Bitwise equality, any NaN matching any NaN."""
    nan = np.isnan(a) & np.isnan(b)
    w = np.uint32 if a.dtype == np.float32 else np.uint64
    return np.all((a.view(w) == b.view(w)) | nan) and np.array_equal(np.isnan(a), np.isnan(b))


def _pair(n_seed):
    x = _doubles(n_seed)
    y = _floats(n_seed + 1)
    m = min(x.size, y.size)
    return x[:m], y[:m]


def test_host_conversions_match_ieee():
    x, y = _pair(11)
    xn, yw, xh, yh = amrmhd.fp_convert(x, y, on_device=False)
    assert _same_bits(xn, _expect_narrow(x))
    assert _same_bits(yw, _expect_widen(y))
    # the harness: the host compiler's casts are numpy's
    with np.errstate(over="ignore", invalid="ignore"):
        assert _same_bits(xh, x.astype(np.float32))
        assert _same_bits(yh, y.astype(np.float64))


def test_ties_round_to_even():
    f = np.array([1.0, 1.0 + 2.0 ** -23, 3.0, 1e30], dtype=np.float32)
    g = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + g.astype(np.float64)) / 2.0
    xn, _, _, _ = amrmhd.fp_convert(mid, np.zeros_like(f), on_device=False)
    even = np.where((f.view(np.uint32) & 1) == 0, f, g)
    assert np.array_equal(xn.view(np.uint32), even.view(np.uint32))


def test_argument_errors():
    with pytest.raises(ValueError):
        amrmhd.fp_convert(np.zeros(3), np.zeros(2, np.float32))
    assert amrmhd.lib().amrmhd_fp_convert(2, 0, None, None, None, None, None, None) != 0
    assert amrmhd.lib().amrmhd_fp_convert(0, 1, None, None, None, None, None, None) != 0
    assert amrmhd.lib().amrmhd_fp_convert(0, 0, None, None, None, None, None, None) == 0


@pytest.mark.gpu
def test_device_conversions_match_instructions_and_host():
    x, y = _pair(23)
    xn, yw, xh, yh = amrmhd.fp_convert(x, y, on_device=True)
    hn, hw, _, _ = amrmhd.fp_convert(x, y, on_device=False)
    assert _same_bits(xn, hn) and _same_bits(yw, hw)
    # against the conversion instructions of the flushed-denormal unit, away
    # from the flushed range (checked against zero above)
    big = np.abs(x) >= TINY
    assert _same_bits(xn[big], xh[big])
    norm = (y.view(np.uint32) & 0x7F800000) != 0
    assert _same_bits(yw[norm], yh[norm])
    assert _same_bits(xn, _expect_narrow(x))
