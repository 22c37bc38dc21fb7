"""Rounding of exact rationals to IEEE-754 binary32 (round to nearest, ties
to the even significand), written out from the format's definition: the
independent reference for the oracle's arithmetic pins."""
from __future__ import annotations

import math
from fractions import Fraction

F32_MAX_EXP = 127
F32_MANT = 23
F32_MIN_EXP = -126  # smallest normal exponent


def round_f32(x: Fraction) -> float:
    """Round an exact rational to the nearest binary32 value, ties to the
    even significand; magnitudes at or above 2^128 - 2^103 (halfway past the
    largest finite value) become infinite."""
    if x == 0:
        return 0.0
    sign = -1.0 if x < 0 else 1.0
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    # quantum of the result: 2^(e - 23) for normals, 2^-149 below them
    q = max(e - F32_MANT, F32_MIN_EXP - F32_MANT)
    scaled = a / (Fraction(2) ** q)
    n = scaled.numerator // scaled.denominator
    rem = scaled - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    v = Fraction(n) * Fraction(2) ** q
    if v >= Fraction(2) ** (F32_MAX_EXP + 1):
        return sign * math.inf
    return sign * float(v)
