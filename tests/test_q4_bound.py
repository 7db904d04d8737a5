"""Error bound behind the 8-bit 4-wide node test (host arithmetic, no GPU).

A quantised plane P = (m + q) s, with quantum s = 2^e, is stored as the frame origin
o' = (m - 2^15) s and the scale S = 2^15 s (both exact in FP32) and evaluated on the device
as fmaf(1 + q 2^-15, S * inv, fl(fl(o' - o) * inv)).  The code 1 + q 2^-15 is exact, the
product S * inv is exact (S is a power of two) and the FMA rounds once (covered, as for
every slab test, by widening tmax by 1 + 2 gamma_3).  The quantiser's outward margin must
cover the rest: the plane the FMA sees before its own rounding,
P_eval = P + (off - (o' - o) inv) / inv, lies within M 2^-22 + s 2^-8 of P whenever
|o| <= M, |m s| <= M and |inv| in [1, 2^64].  The check runs the FP32 steps in numpy (IEEE
round-to-nearest) and measures the displacement exactly with fractions, on random and
extreme cases.
"""
from fractions import Fraction

import numpy as np


def _displacement(m, e, o, inv):
    s = Fraction(2) ** e
    o_shift = np.float32(float((m - 2 ** 15) * s))
    assert Fraction(float(o_shift)) == (m - 2 ** 15) * s          # the stored origin is exact
    scale = np.float32(float(2 ** 15 * s))
    assert Fraction(float(scale)) == 2 ** 15 * s                  # and so is the stored scale
    diff = np.float32(o_shift - np.float32(o))
    off = np.float32(diff * np.float32(inv))
    assert np.isfinite(off)
    exact = (Fraction(float(o_shift)) - Fraction(float(np.float32(o)))) * Fraction(float(np.float32(inv)))
    return abs((Fraction(float(off)) - exact) / Fraction(float(np.float32(inv)))), s


def _bound(s, big):
    return Fraction(big) * Fraction(2) ** -22 + s * Fraction(2) ** -8


def test_one_fma_plane_error_within_quantiser_margin():
    rng = np.random.default_rng(1806)
    worst = 0.0
    for big in (1280.0, 2560.0, 1.0e4, 3.0e5):
        for _ in range(1500):
            e = int(rng.integers(-12, 9))
            s = 2.0 ** e
            lim = int(min(big / s, 2 ** 23 - 1))
            m = int(rng.integers(-lim, lim + 1))
            o = float(rng.choice([rng.uniform(-big, big), big, -big, 0.0, m * s]))
            d = float(rng.choice([rng.uniform(-1.0, 1.0), 2.0 ** -64, -(2.0 ** -64), 1.0, -1.0,
                                  rng.uniform(-1e-6, 1e-6)]))
            inv = float(np.clip(np.float32(1.0) / np.float32(d if d != 0.0 else 1e-30), -2.0 ** 64, 2.0 ** 64))
            disp, sf = _displacement(m, e, o, inv)
            bound = _bound(sf, big)
            assert disp <= bound, (big, e, m, o, inv, float(disp), float(bound))
            worst = max(worst, float(disp / bound))
    assert worst > 0.25          # the cases come close to the bound, so a much smaller margin would fail


def test_margin_is_a_small_fraction_of_a_leaf_level_quantum():
    # nodes just above the leaves of a 256^3 foam of 10 nm voxels (M about 2590 nm) span
    # 10-40 nm, so their quantum is 2^-5-2^-3 nm: the quantiser's margin, twice the decode
    # bound, is below 1/16 of it, where the 0x4B0000qq decode needed two whole quanta
    big = 2590.0
    for span in (10.0, 20.0, 40.0):
        s = Fraction(2) ** int(np.floor(np.log2(span / 250.0)))
        assert 2 * _bound(s, big) < s / 16
        for m in (0, int(big / float(s)) - 300):
            disp, sf = _displacement(m, int(np.log2(float(s))), big, -1.0)
            assert disp <= _bound(sf, big)


def test_shifted_origin_stays_finite_at_the_format_limits():
    # largest quantum (2^40), frame at the far end of its range, |1/d| at the clamp: the offset
    # stays finite and moves the plane by at most |o' - o| 2^-23
    for m in (-(2 ** 23 - 1), 0, 2 ** 23 - 1):
        for o, inv in ((0.0, 2.0 ** 64), (3.0e5, -(2.0 ** 64))):
            disp, sf = _displacement(m, 40, o, inv)
            assert disp <= (abs(m - 2 ** 15) * sf + Fraction(o)) * Fraction(2) ** -23
