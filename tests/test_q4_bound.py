"""Error bound behind the 8-bit 4-wide node test (host arithmetic, no GPU).

A quantised plane P = o' + (2^23 + q) s, with o' = (m - 2^23) s exact in FP32,
is evaluated on the device as fmaf(2^23 + q, s * inv, fl(fl(o' - o) * inv)).
The product s * inv is exact (s is a power of two) and the FMA rounds once
(covered, as for every slab test, by widening tmax by 1 + 2 gamma_3).  The
quantiser's outward margin must cover the rest: the plane the FMA sees before
its own rounding, P_eval = P + (off - (o' - o) inv) / inv, lies within
s + M 2^-22 of P whenever |o| <= M, |m s| <= M and |inv| in [1, 2^64].  The
check runs the FP32 steps in numpy (IEEE round-to-nearest) and measures the
displacement exactly with fractions, on random and extreme cases.
"""
from fractions import Fraction

import numpy as np


def _displacement(m, e, o, inv):
    s = Fraction(2) ** e
    o_shift = np.float32(float((m - 2 ** 23) * s))
    assert Fraction(float(o_shift)) == (m - 2 ** 23) * s          # the stored origin is exact
    diff = np.float32(o_shift - np.float32(o))
    off = np.float32(diff * np.float32(inv))
    assert np.isfinite(off)
    exact = (Fraction(float(o_shift)) - Fraction(float(np.float32(o)))) * Fraction(float(np.float32(inv)))
    return abs((Fraction(float(off)) - exact) / Fraction(float(np.float32(inv)))), s


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
            bound = sf + Fraction(big) * Fraction(2) ** -22
            assert disp <= bound, (big, e, m, o, inv, float(disp), float(bound))
            worst = max(worst, float(disp / bound))
    assert worst > 0.5           # the cases come close to the bound, so a smaller margin would fail


def test_shifted_origin_stays_finite_at_the_format_limits():
    # largest quantum (2^40), frame at the far end of its range, |1/d| at the clamp
    for m in (-(2 ** 23 - 1), 0, 2 ** 23 - 1):
        disp, sf = _displacement(m, 40, 0.0, 2.0 ** 64)
        assert disp <= sf
        disp, sf = _displacement(m, 40, 3.0e5, -(2.0 ** 64))
        assert disp <= sf + Fraction(3.0e5) * Fraction(2) ** -22
