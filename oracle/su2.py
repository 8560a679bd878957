"""SU(2) representation data for the oracle, written out from explicit Clebsch-Gordan tensors.

Test infrastructure (see the package header).  All spins are passed as twice their value
(``tj = 2j``, ``tm = 2m``).

* ``cg``: Clebsch-Gordan coefficient <j1 m1; j2 m2 | J M> in the Condon-Shortley phase
  convention, from Racah's closed formula (textbook).  These are the components of the
  splitting tensor X^{ab}_c (Sec. 4.1: the splitting-tensor components are the CG
  coefficients).  Pinned by orthonormality/completeness, the j (x) 1/2 closed forms and
  <j m; j -m | 0 0> = (-1)^(j-m)/sqrt(2j+1) (Sec. 4.2, X^{a abar}_I = (1 (x) Z_a) eta_a/sqrt(d_a)).
* ``zmat``: the duality isomorphism Z_j : (V^j)* -> V^j with (Z_j)_{m',m} = (-1)^(j-m) delta_{m',-m}
  (reading of Sec. 4.2 fixed by the relation above; pinned by Z^T = chi Z with chi_j = (-1)^(2j),
  Sec. 5.4).
* ``sixj_exact`` / ``fsymbol_exact``: the 6j symbol from Racah's formula and
  F^{j1 j2 j3}_{j4}[j5, j6] = sqrt(d5 d6) (-1)^(j1+j2+j3+j4) {j1 j2 j5; j3 j4 j6} (eq. SU2FSymbol),
  exact and correctly rounded.  Pinned against ``fsymbol_from_cg`` (projection of the associator,
  Sec. 5.4) and the pentagon equation.
* ``fsymbol_from_cg`` / ``rsymbol_from_cg``: F and R obtained by projecting explicit CG trees
  (Sec. 5.4, the Rep G construction of F and R).
"""

from fractions import Fraction
from functools import lru_cache

import numpy as np

from .exact import fact, signed_sqrt

__all__ = [
    "cg", "cg_exact", "cg_tensor", "zmat", "sixj_exact", "fsymbol_exact", "fsymbol_from_cg",
    "rsymbol_from_cg", "triangle", "dim",
]


def dim(tj: int) -> int:
    return tj + 1


def triangle(ta: int, tb: int, tc: int) -> bool:
    """N^{ab}_c for SU(2) (eq. SU2NSymbol): |a-b| <= c <= a+b and a+b+c integer."""
    return abs(ta - tb) <= tc <= ta + tb and (ta + tb + tc) % 2 == 0


@lru_cache(maxsize=None)
def cg_exact(tj1: int, tm1: int, tj2: int, tm2: int, tJ: int, tM: int):
    """Return (sign, square) with <j1 m1; j2 m2|J M> = sign * sqrt(square), exactly."""
    if tm1 + tm2 != tM or not triangle(tj1, tj2, tJ):
        return 0, Fraction(0)
    for tj, tm in ((tj1, tm1), (tj2, tm2), (tJ, tM)):
        if abs(tm) > tj or (tj + tm) % 2:
            return 0, Fraction(0)
    h = lambda x: x // 2  # all arguments below are even by the checks above
    pref = Fraction(
        (tJ + 1) * fact(h(tj1 + tj2 - tJ)) * fact(h(tj1 - tj2 + tJ)) * fact(h(-tj1 + tj2 + tJ)),
        fact(h(tj1 + tj2 + tJ) + 1),
    )
    pref *= (fact(h(tj1 + tm1)) * fact(h(tj1 - tm1)) * fact(h(tj2 + tm2)) * fact(h(tj2 - tm2))
             * fact(h(tJ + tM)) * fact(h(tJ - tM)))
    s = Fraction(0)
    k = 0
    while True:
        args = [k, h(tj1 + tj2 - tJ) - k, h(tj1 - tm1) - k, h(tj2 + tm2) - k,
                h(tJ - tj2 + tm1) + k, h(tJ - tj1 - tm2) + k]
        if args[1] < 0 or args[2] < 0 or args[3] < 0:
            break
        if min(args) >= 0:
            den = 1
            for a in args:
                den *= fact(a)
            s += Fraction((-1) ** k, den)
        k += 1
    if s == 0:
        return 0, Fraction(0)
    return (1 if s > 0 else -1), pref * s * s


@lru_cache(maxsize=None)
def cg(tj1: int, tm1: int, tj2: int, tm2: int, tJ: int, tM: int) -> float:
    sgn, sq = cg_exact(tj1, tm1, tj2, tm2, tJ, tM)
    return 0.0 if sgn == 0 else signed_sqrt(sgn, sq)


@lru_cache(maxsize=None)
def cg_tensor(tj1: int, tj2: int, tJ: int) -> np.ndarray:
    """Splitting tensor X^{j1 j2}_J as an array [m1, m2, M] (index = (tm + tj)/2, m ascending)."""
    out = np.zeros((tj1 + 1, tj2 + 1, tJ + 1))
    if not triangle(tj1, tj2, tJ):
        return out
    for i1 in range(tj1 + 1):
        tm1 = 2 * i1 - tj1
        for i2 in range(tj2 + 1):
            tm2 = 2 * i2 - tj2
            tM = tm1 + tm2
            if abs(tM) <= tJ:
                out[i1, i2, (tM + tJ) // 2] = cg(tj1, tm1, tj2, tm2, tJ, tM)
    out.setflags(write=False)
    return out


@lru_cache(maxsize=None)
def zmat(tj: int) -> np.ndarray:
    """(Z_j)[m', m] = (-1)^(j-m) delta_{m', -m}; rows index V^j, columns the dual basis."""
    d = tj + 1
    z = np.zeros((d, d))
    for i in range(d):  # column i <-> m = (2i - tj)/2 ; row tj - i <-> m' = -m
        tm = 2 * i - tj
        z[tj - i, i] = (-1) ** ((tj - tm) // 2)
    z.setflags(write=False)
    return z


def _delta_sq(ta: int, tb: int, tc: int) -> Fraction:
    h = lambda x: x // 2
    return Fraction(fact(h(ta + tb - tc)) * fact(h(ta - tb + tc)) * fact(h(-ta + tb + tc)),
                    fact(h(ta + tb + tc) + 1))


@lru_cache(maxsize=None)
def sixj_exact(t1: int, t2: int, t3: int, t4: int, t5: int, t6: int):
    """{j1 j2 j3; j4 j5 j6} by Racah's formula as (sign, square), exact.

    Non-zero only if the triads (j1 j2 j3), (j1 j5 j6), (j4 j2 j6), (j4 j5 j3) are admissible.
    """
    triads = ((t1, t2, t3), (t1, t5, t6), (t4, t2, t6), (t4, t5, t3))
    if not all(triangle(*t) for t in triads):
        return 0, Fraction(0)
    pre = Fraction(1)
    for t in triads:
        pre *= _delta_sq(*t)
    a = [sum(t) // 2 for t in triads]                    # t >= each triad sum
    b = [(t1 + t2 + t4 + t5) // 2, (t2 + t3 + t5 + t6) // 2, (t3 + t1 + t6 + t4) // 2]
    s = Fraction(0)
    for t in range(max(a), min(b) + 1):
        den = 1
        for x in a:
            den *= fact(t - x)
        for y in b:
            den *= fact(y - t)
        s += Fraction((-1) ** t * fact(t + 1), den)
    if s == 0:
        return 0, Fraction(0)
    return (1 if s > 0 else -1), pre * s * s


@lru_cache(maxsize=None)
def fsymbol_exact(t1: int, t2: int, t3: int, t4: int, t5: int, t6: int) -> float:
    """F^{j1 j2 j3}_{j4}[j5; j6] of eq. SU2FSymbol, correctly rounded from its exact value.

    j5 is the coupling of (j1 j2) in the left-to-right tree, j6 the coupling of (j2 j3).
    """
    sgn, sq = sixj_exact(t1, t2, t5, t3, t4, t6)
    if sgn == 0:
        return 0.0
    phase = (t1 + t2 + t3 + t4) // 2
    if phase % 2:
        sgn = -sgn
    return signed_sqrt(sgn, sq * (t5 + 1) * (t6 + 1))


@lru_cache(maxsize=None)
def _left_tree(ta, tb, tc, te, td):
    # ((a b)_e c)_d as array [ma, mb, mc, md]
    return np.einsum("xye,ezd->xyzd", cg_tensor(ta, tb, te), cg_tensor(te, tc, td))


@lru_cache(maxsize=None)
def _right_tree(ta, tb, tc, tf, td):
    # (a (b c)_f)_d as array [ma, mb, mc, md]
    return np.einsum("yzf,xfd->xyzd", cg_tensor(tb, tc, tf), cg_tensor(ta, tf, td))


def fsymbol_from_cg(ta, tb, tc, td, te, tf) -> float:
    """F^{abc}_d[e; f] = <(a (b c)_f)_d | ((a b)_e c)_d> / d_d (Sec. 5.4, projection of eq. associator)."""
    if not (triangle(ta, tb, te) and triangle(te, tc, td) and triangle(tb, tc, tf)
            and triangle(ta, tf, td)):
        return 0.0
    return float(np.sum(_left_tree(ta, tb, tc, te, td) * _right_tree(ta, tb, tc, tf, td)) / (td + 1))


def rsymbol_from_cg(ta, tb, tc) -> float:
    """R^{ab}_c from tau_{a,b} X^{ab}_c = R^{ab}_c X^{ba}_c (eq. braiding), with tau the plain swap."""
    if not triangle(ta, tb, tc):
        return 0.0
    x = cg_tensor(ta, tb, tc)
    y = cg_tensor(tb, ta, tc)
    swapped = np.transpose(x, (1, 0, 2))  # components of tau X^{ab}_c in the (b, a) order
    return float(np.sum(swapped * y) / (tc + 1))
