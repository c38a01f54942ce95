"""Host replay of the space-variant kernel's fixed-point arithmetic.

The kernel centres each tile (f~ = f - c, c the middle of the extended tile's
range, h = max |f~|), stores every plane value v as round(v 2^k) through one
FP32 FMA against 1.5 * 2^23 (the result lies in [2^23, 2^24), where the FP32
spacing is 1), keeps the raw bit patterns in wrapping 32-bit summed-area
tables and removes (box area) x (the constant's bit pattern) from each box
sum.  The exponent is 21 or 20 for the plain planes (|v| <= 1) and a per-tile
power of two for the f~-weighted ones (|v| <= h), chosen so that every rounded
value stays below 2^21 and every box of the largest size sums below 2^31.
These tests replay each of those steps in numpy (IEEE single precision where
the kernel uses it) and check them against exact integer arithmetic."""
from fractions import Fraction

import numpy as np

M = np.float32(12582912.0)  # 1.5 * 2^23
MBITS = int(np.array([M]).view(np.uint32)[0])
CAP = 2 ** 21  # largest rounded magnitude the kernel allows


def _nbox(rm):
    return (2 * rm + 1) ** 2


def _plain_exponent(nbox):
    k = 21
    while k > 0 and 2.0 ** k * nbox >= 0.999 * 2.0 ** 31:
        k -= 1
    return k


def _weighted_exponent(h, nbox):
    # FP32 steps of the kernel: lim = cap / max(h, 1e-30); k = floor(log2(lim))
    cap = np.float32(min(0.999 * 2.0 ** 31 / nbox, float(CAP)))
    lim = np.float32(cap / np.maximum(np.float32(h), np.float32(1e-30)))
    k = int((np.array([lim]).view(np.int32)[0] >> 23) - 127)
    return min(max(k, -60), 60), float(cap)


def _fma_round(v, k):
    """fma(v, 2^k, 1.5 * 2^23) in FP32, returned as (bit pattern - MBITS).
    v * 2^k is exact; v * 2^k + M is exact in FP64 for the magnitudes used,
    so one rounding to FP32 is the FMA's single rounding."""
    v = np.asarray(v, dtype=np.float32).astype(np.float64)
    th = (v * 2.0 ** k + float(M)).astype(np.float32)
    return th.view(np.uint32).astype(np.int64) - MBITS


def _round_half_even(v, k):
    fr = Fraction(float(v)) * Fraction(2) ** k
    fl = fr.numerator // fr.denominator
    rem = fr - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return fl


def test_plain_exponents_keep_box_sums_in_32_bits():
    assert [_plain_exponent(_nbox(rm)) for rm in (4, 8, 16)] == [21, 21, 20]
    for rm in (4, 8, 16):
        k = _plain_exponent(_nbox(rm))
        assert 2 ** k <= CAP and _nbox(rm) * 2 ** k < 2 ** 31


def test_fma_against_the_constant_is_exact_rounding():
    rng = np.random.default_rng(0)
    for k in (21, 20, 13, 15, -3):
        lim = CAP / 2.0 ** k
        tie = 2.0 ** (-k - 1)
        v = np.concatenate([
            rng.uniform(-lim, lim, 4000), rng.uniform(-1e-3, 1e-3, 500) * lim,
            [0.0, -0.0, lim, -lim, tie, 3 * tie, 5 * tie, -3 * tie, -5 * tie, 1e-30, -1e-30],
        ]).astype(np.float32)
        got = _fma_round(v, k)
        for i in range(len(v)):
            assert got[i] == _round_half_even(v[i], k), (k, float(v[i]))
        assert np.abs(got).max() <= CAP


def test_centring_bounds_every_value_and_the_weighted_exponent_fits():
    rng = np.random.default_rng(1)
    tiles = [rng.integers(0, 256, 300).astype(np.float32),             # u8 data
             rng.uniform(0, 255, 300).astype(np.float32),
             (1e6 + rng.uniform(0, 1, 300)).astype(np.float32),        # narrow range, large offset
             rng.uniform(-3e4, 5e4, 300).astype(np.float32),
             np.full(300, 17.25, np.float32)]                          # constant tile
    for f in tiles:
        mn, mx = f.min(), f.max()
        c = np.float32(mn + np.float32(0.5) * np.float32(mx - mn))
        h = np.float32(max(np.float32(mx - c), np.float32(c - mn)))
        ft = (f - c).astype(np.float32)
        assert np.abs(ft).max() <= h
        for rm in (4, 8, 16):
            k, cap = _weighted_exponent(h, _nbox(rm))
            # every f~ cos / f~ sin value rounds below the cap, and a box of them sums below 2^31
            assert float(h) * 2.0 ** k <= cap * (1 + 2 ** -20)
            assert _nbox(rm) * cap < 2 ** 31 and cap <= CAP
            if h > 0:  # the largest such power of two (up to the FP32 division's rounding)
                assert float(h) * 2.0 ** (k + 1) > cap * (1 - 2 ** -20)


def test_biased_wrapping_tables_give_exact_box_sums():
    # steps 1-3 of the kernel in uint32: running sums of the raw bit patterns
    # along rows, then down columns; a box sum minus (area x MBITS) is exact
    rng = np.random.default_rng(2)
    E = 64
    # (exponent, largest half-width it serves); the constant planes at +-cap
    # make every prefix sum wrap and every box sum reach its largest value
    for k, rmax, kind in [(21, 8, "uniform"), (21, 8, "max"), (20, 16, "uniform"),
                          (20, 16, "min"), (13, 16, "uniform")]:
        # the largest rounded magnitude at this box size: 2^k for the plain
        # planes (|v| <= 1), the cap for the weighted ones
        bound = min(float(CAP), 0.999 * 2.0 ** 31 / _nbox(rmax))
        lim = np.float32(bound / 2.0 ** k)
        if kind == "uniform":
            v = rng.uniform(-lim, lim, (E, E)).astype(np.float32)
        else:
            v = np.full((E, E), lim if kind == "max" else -lim, np.float32)
        q = _fma_round(v, k)
        raw = (q + MBITS).astype(np.uint32)  # the FP32 bit patterns the kernel adds
        T = np.zeros((E + 1, E + 1), np.uint32)
        with np.errstate(over="ignore"):
            T[1:, 1:] = np.cumsum(np.cumsum(raw, axis=1, dtype=np.uint32), axis=0, dtype=np.uint32)
        for _ in range(300):
            r = int(rng.integers(0, rmax + 1))
            i, j = rng.integers(r, E - r, 2)
            a0, a1, b0, b1 = i - r, i + r + 1, j - r, j + r + 1
            with np.errstate(over="ignore"):
                s = (T[a1, b1] - T[a0, b1] - T[a1, b0] + T[a0, b0]
                     - np.uint32(((2 * r + 1) ** 2 * MBITS) % 2 ** 32))
            exact = int(q[a0:a1, b0:b1].sum())
            assert int(np.array([s]).view(np.int32)[0]) == exact
            assert abs(exact) < 2 ** 31
