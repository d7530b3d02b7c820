"""Pins of the oracle's cast storage formats (float32 / float16 as in the Compression
Configuration, bfloat16 as one more cast) against library routines and exhaustive enumeration:
every pair of neighbouring representable values is built from its bit pattern, and the values
on both sides of, and exactly at, their midpoint must round to the right neighbour (ties to even)."""
import numpy as np
import pytest


def _neighbour_checks(orc, fmt, vals_from_bits, nbits_max):
    bits = np.arange(0, nbits_max, dtype=np.int64)
    a = vals_from_bits(bits)
    b = vals_from_bits(bits + 1)
    mid = (a + b) / 2.0  # exact: both have few significant bits
    below = np.nextafter(mid, -np.inf)
    above = np.nextafter(mid, np.inf)
    even = np.where(bits % 2 == 0, a, b)
    for sign in (1.0, -1.0):
        assert np.array_equal(orc.cast_decode(orc.cast_encode(sign * a, fmt), fmt), sign * a)
        assert np.array_equal(orc.cast_decode(orc.cast_encode(sign * mid, fmt), fmt), sign * even)
        assert np.array_equal(orc.cast_decode(orc.cast_encode(sign * below, fmt), fmt), sign * a)
        assert np.array_equal(orc.cast_decode(orc.cast_encode(sign * above, fmt), fmt), sign * b)


def test_bf16_exhaustive(orc):
    def vals(bits):
        return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)

    _neighbour_checks(orc, orc.BF16, vals, 0x7F7F)  # up to the largest finite bfloat16
    # bit patterns are the top half of the binary32 pattern
    x = np.array([1.0, -2.0, 0.15625, 2.0 ** -133])
    assert list(orc.cast_encode(x, orc.BF16)) == [0x3F80, 0xC000, 0x3E20, 0x0001]
    top = vals(np.array([0x7F7F]))[0]
    ulp = top - vals(np.array([0x7F7E]))[0]
    assert np.isinf(orc.cast_round(top + ulp / 2, orc.BF16))


def test_fp16_exhaustive_and_numpy(orc):
    def vals(bits):
        return bits.astype(np.uint16).view(np.float16).astype(np.float64)

    _neighbour_checks(orc, orc.FP16, vals, 0x7BFF)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(200000) * np.exp2(rng.integers(-30, 15, 200000))
    assert np.array_equal(orc.cast_encode(x, orc.FP16), x.astype(np.float16).view(np.uint16))
    assert np.array_equal(orc.cast_decode(x.astype(np.float16).view(np.uint16), orc.FP16),
                          x.astype(np.float16).astype(np.float64))


def test_fp32_numpy_and_ties(orc):
    rng = np.random.default_rng(6)
    x = rng.standard_normal(200000) * np.exp2(rng.integers(-160, 120, 200000))
    assert np.array_equal(orc.cast_encode(x, orc.FP32), x.astype(np.float32).view(np.uint32))
    bits = rng.integers(0, 0x7F7FFFFF, 100000)

    def vals(b):
        return b.astype(np.uint32).view(np.float32).astype(np.float64)

    a, b = vals(bits), vals(bits + 1)
    mid = (a + b) / 2.0
    even = np.where(bits % 2 == 0, a, b)
    assert np.array_equal(orc.cast_decode(orc.cast_encode(mid, orc.FP32), orc.FP32), even)
    assert np.array_equal(mid.astype(np.float32).astype(np.float64), even)


@pytest.mark.parametrize("fmt", [0, 1, 2, 3])
def test_signed_zero_and_roundtrip(orc, fmt):
    x = np.array([0.0, -0.0, 1.0, -1.0, 0.5])
    d = orc.cast_decode(orc.cast_encode(x, fmt), fmt)
    assert np.array_equal(np.signbit(d), np.signbit(x))
    assert np.array_equal(d, x)
