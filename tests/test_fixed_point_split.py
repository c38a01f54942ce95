"""The space-variant kernel stores round(v * 2^26) as hi * 2^20 + lo, computed
with FP32 additions (adding 1.5 * 2^23 rounds a float below 2^22 to the
nearest integer, ties to even).  This test replays that sequence of IEEE
single-precision operations in numpy and checks it against exact rational
rounding, and the ranges that keep every 33 x 33 box sum of either half
inside 32 bits."""
from fractions import Fraction

import numpy as np

M = np.float32(12582912.0)  # 1.5 * 2^23
MBITS = int(np.array([M]).view(np.int32)[0])


def _split(v):
    v = np.asarray(v, dtype=np.float32)
    x = (v * np.float32(2.0 ** 26)).astype(np.float32)
    th = ((x * np.float32(2.0 ** -20)).astype(np.float32) + M).astype(np.float32)
    hi = th.view(np.int32).astype(np.int64) - MBITS
    hf = (th - M).astype(np.float32)
    # the kernel uses one FMA; the product is exact, so the separate steps agree
    lo_f = (x - (hf * np.float32(2.0 ** 20)).astype(np.float32)).astype(np.float32)
    lo = (lo_f + M).astype(np.float32).view(np.int32).astype(np.int64) - MBITS
    return hi, lo


def _round_half_even(v):
    fr = Fraction(float(v)) * 2 ** 26
    fl = fr.numerator // fr.denominator
    rem = fr - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return fl


def test_split_is_exact_rounding():
    rng = np.random.default_rng(0)
    tie = 2.0 ** -27
    v = np.concatenate([
        rng.uniform(-255, 255, 6000), rng.uniform(-1, 1, 6000), rng.uniform(-1e-4, 1e-4, 2000),
        [0.0, -0.0, 255.0, -255.0, 1.0, -1.0, 1e-30, -1e-30, tie, 3 * tie, 5 * tie, -3 * tie,
         2.0 ** -6 + tie, 127.99998, -127.99998]]).astype(np.float32)
    hi, lo = _split(v)
    for k in range(len(v)):
        assert hi[k] * 2 ** 20 + lo[k] == _round_half_even(v[k]), float(v[k])


def test_split_ranges_keep_box_sums_in_32_bits():
    v = np.linspace(-255, 255, 200001).astype(np.float32)
    hi, lo = _split(v)
    assert np.abs(hi).max() <= 16320 and np.abs(lo).max() <= 2 ** 19
    n = 33 * 33  # the largest box
    assert n * 16320 < 2 ** 31 and n * 2 ** 19 < 2 ** 31
