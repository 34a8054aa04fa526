"""The fused kernel normalises a cell without a division per bin: with r = RN(1/n) it forms
q0 = RN(h r), rem = fma(-q0, n, h) (exact) and q = RN(rem r + q0).  This must equal the IEEE
single quotient RN(h / n) that the oracle computes, for every count pair a cell can hold
(0 <= h <= n <= 64, since a cell has 8 x 8 pixels).  Checked exhaustively here in exact
rational arithmetic, so the kernel's normalised rows can be compared bit for bit."""
import math
from fractions import Fraction

import numpy as np


def _rn32(fr):
    """Round a rational to the nearest float32 (ties to even), exactly."""
    if fr == 0:
        return np.float32(0.0)
    s = -1 if fr < 0 else 1
    a = abs(fr)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    q = a / Fraction(2) ** (e - 23)
    fl = q.numerator // q.denominator
    rem = q - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return np.float32(s * fl * 2.0 ** (e - 23))


def test_rn32_matches_numpy_on_products():
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b = np.float32(rng.random()), np.float32(rng.random() * 64)
        want = np.float32(a * b)
        assert _rn32(Fraction(float(a)) * Fraction(float(b))) == want


def test_reciprocal_correction_is_the_ieee_quotient():
    for n in range(1, 65):
        r = np.float32(1.0) / np.float32(n)
        for h in range(0, n + 1):
            q0 = np.float32(np.float32(h) * r)
            rem = _rn32(Fraction(h) - Fraction(float(q0)) * n)
            q = _rn32(Fraction(float(rem)) * Fraction(float(r)) + Fraction(float(q0)))
            want = np.float32(h) / np.float32(n)
            assert q.view(np.uint32) == want.view(np.uint32), (h, n)
