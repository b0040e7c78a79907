"""The step divides the pressure moment by 3 as q0 = RN(x c), r = x - 3 q0
(exact, as an FMA forms it), q = RN(q0 + r c) with c = RN(1/3): one residual
correction in FMA form, after Markstein's method for correctly rounded
division.  This checks, in exact rational arithmetic where binary64 cannot
decide, that the result is the correctly rounded x/3: every FP32 mantissa
of one binade (the rounding pattern repeats in every binade of normal
numbers), and a seeded sample of FP64 values over 120 binades."""
import random
from fractions import Fraction

import numpy as np


def _rn32(fr):
    """Round a rational to the nearest float32, ties to even."""
    f = np.float32(float(fr))
    cands = [f, np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(-np.inf))]
    return min(cands, key=lambda v: (abs(Fraction(float(v)) - fr),
                                     int(np.frombuffer(np.float32(v).tobytes(), np.uint32)[0]) & 1))


def test_fp32_division_by_three_is_correctly_rounded():
    c = np.float32(1.0) / np.float32(3.0)
    m = np.arange(2 ** 23, dtype=np.int64)
    x = ((1.0 + m / 2.0 ** 23)).astype(np.float32)  # every mantissa of [1, 2)
    x64 = x.astype(np.float64)
    q0 = (x64 * np.float64(c)).astype(np.float32)  # the product is exact in binary64
    r = x64 - 3.0 * q0.astype(np.float64)           # exact
    assert np.all(np.abs(r) < 2.0 ** -20)           # r fits in float32 exactly (FMA output)
    assert np.all(r.astype(np.float32).astype(np.float64) == r)
    q = (q0.astype(np.float64) + r * np.float64(c)).astype(np.float32)
    ref = (x64 / 3.0).astype(np.float32)
    # both sides above may round twice (binary64, then float32): decide the
    # values where they differ exactly
    bad = 0
    for i in np.nonzero(q != ref)[0]:
        exact = _rn32(Fraction(float(x[i])) / 3)
        fma = _rn32(Fraction(float(q0[i])) + Fraction(float(r[i])) * Fraction(float(c)))
        bad += exact != fma
    assert bad == 0


def test_fp64_division_by_three_is_correctly_rounded_sampled():
    rng = random.Random(3)
    c = 1.0 / 3.0
    for _ in range(20000):
        x = rng.uniform(1.0, 2.0) * 2.0 ** rng.randint(-60, 60)
        q0 = x * c
        r = Fraction(x) - 3 * Fraction(q0)
        assert Fraction(float(r)) == r  # the FMA's x - 3 q0 is exact
        q = float(Fraction(q0) + r * Fraction(c))  # one rounding, as the FMA
        assert q == float(Fraction(x) / 3)
