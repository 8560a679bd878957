"""Exact rational helpers for the oracle (test infrastructure).

Symbols of SU(2) that the oracle needs exactly (Clebsch-Gordan coefficients, 6j symbols,
F-symbols) are all of the form  sign * sqrt(q)  with q a non-negative rational.  This module
turns such a value into the correctly rounded IEEE double, using Python's arbitrary-precision
integers only.
"""

from fractions import Fraction
from math import factorial, isqrt

__all__ = ["sqrt_rational", "signed_sqrt", "fact"]


def fact(n: int) -> int:
    if n < 0:
        raise ValueError("negative factorial argument")
    return factorial(n)


def sqrt_rational(q: Fraction) -> float:
    """Correctly rounded (round-to-nearest-even) double of sqrt(q) for a rational q >= 0."""
    q = Fraction(q)
    if q < 0:
        raise ValueError("sqrt of a negative rational")
    if q == 0:
        return 0.0
    p, d = q.numerator, q.denominator
    # Choose k so that r = floor(sqrt(p/d * 4^k)) has at least 64 significant bits.
    k = max(0, 140 - (p.bit_length() - d.bit_length()) // 2)
    n = (p << (2 * k)) // d
    r = isqrt(n)
    exact = (r * r * d) == (p << (2 * k))
    # Append a sticky bit so that the final int/int true division (correctly rounded in
    # CPython) sees "strictly above" whenever the discarded tail is non-zero.
    rs = (r << 1) | (0 if exact else 1)
    return rs / (1 << (k + 1))


def signed_sqrt(sign: int, q: Fraction) -> float:
    v = sqrt_rational(q)
    return -v if sign < 0 else v
