"""Pins of the oracle's SU(2) representation data and of its generic consistency checkers.

Every check compares the oracle against something the paper or the mathematics fixes, not
against a retyping of the oracle's own formula.
"""

import cmath
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from golden_io import lines, value
from oracle import su2
from oracle.exact import sqrt_rational

JMAX2 = 8  # 2j up to 4, the largest spin of the SU(2) workloads


def spins(maxtj=JMAX2):
    return range(0, maxtj + 1)


# ------------------------------------------------------------------ exact arithmetic
def test_sqrt_rational_correct_rounding():
    for q in [Fraction(2), Fraction(1, 3), Fraction(7, 10), Fraction(10**30 + 7, 3**40)]:
        v = sqrt_rational(q)
        # v is the correctly rounded value iff the true sqrt lies within half an ulp of v
        lo, hi = Fraction(v) - Fraction(math.ulp(v)) / 2, Fraction(v) + Fraction(math.ulp(v)) / 2
        assert lo * lo <= q <= hi * hi
    assert sqrt_rational(Fraction(9, 4)) == 1.5
    assert sqrt_rational(Fraction(2)) == math.sqrt(2.0)  # IEEE sqrt is correctly rounded


# ------------------------------------------------------------------ Clebsch-Gordan
def test_cg_half_closed_forms():
    """j (x) 1/2 coefficients against the textbook closed forms (all j <= 4)."""
    for tj in spins():
        for tM in range(-(tj + 1), tj + 2, 2):
            # J = j + 1/2
            tJ = tj + 1
            a = su2.cg(tj, tM - 1, 1, 1, tJ, tM) if abs(tM - 1) <= tj else 0.0
            b = su2.cg(tj, tM + 1, 1, -1, tJ, tM) if abs(tM + 1) <= tj else 0.0
            assert a == pytest.approx(math.sqrt((tj + tM + 1) / 2 / (tj + 1)) if abs(tM - 1) <= tj else 0.0, abs=1e-15)
            assert b == pytest.approx(math.sqrt((tj - tM + 1) / 2 / (tj + 1)) if abs(tM + 1) <= tj else 0.0, abs=1e-15)
            if tj >= 1 and abs(tM) <= tj - 1:
                tJ = tj - 1
                c = su2.cg(tj, tM + 1, 1, -1, tJ, tM)
                d = su2.cg(tj, tM - 1, 1, 1, tJ, tM)
                assert c == pytest.approx(math.sqrt((tj + tM + 1) / 2 / (tj + 1)), abs=1e-15)
                assert d == pytest.approx(-math.sqrt((tj - tM + 1) / 2 / (tj + 1)), abs=1e-15)


def test_cg_table_values():
    s = math.sqrt
    assert su2.cg(2, 2, 2, -2, 0, 0) == pytest.approx(1 / s(3))
    assert su2.cg(2, 0, 2, 0, 0, 0) == pytest.approx(-1 / s(3))
    assert su2.cg(2, 2, 2, -2, 2, 0) == pytest.approx(1 / s(2))
    assert su2.cg(2, 0, 2, 0, 2, 0) == 0.0
    assert su2.cg(2, 2, 2, -2, 4, 0) == pytest.approx(1 / s(6))
    assert su2.cg(2, 0, 2, 0, 4, 0) == pytest.approx(s(2 / 3))
    assert su2.cg(1, 1, 1, -1, 0, 0) == pytest.approx(1 / s(2))
    assert su2.cg(1, -1, 1, 1, 0, 0) == pytest.approx(-1 / s(2))


def test_cg_singlet_matches_z():
    """X^{a abar}_I = (1 (x) Z_a) eta_a / sqrt(d_a)  (Sec. 4.2) fixes Z against the CG singlet."""
    for tj in spins():
        x = su2.cg_tensor(tj, tj, 0)[:, :, 0]
        z = su2.zmat(tj)
        # (1 (x) Z) eta = sum_m |m> (x) Z<m|  ->  component [m, m'] = Z[m', m]
        assert np.allclose(x, z.T / math.sqrt(tj + 1), atol=1e-15)


def test_cg_orthonormal_complete():
    for tj1, tj2 in itertools.product(spins(6), spins(6)):
        d1, d2 = tj1 + 1, tj2 + 1
        cols = []
        for tJ in range(abs(tj1 - tj2), tj1 + tj2 + 1, 2):
            x = su2.cg_tensor(tj1, tj2, tJ).reshape(d1 * d2, tJ + 1)
            cols.append(x)
        u = np.concatenate(cols, axis=1)
        assert u.shape == (d1 * d2, d1 * d2)
        assert np.allclose(u.T @ u, np.eye(d1 * d2), atol=1e-14)


def _jmats(tj):
    d = tj + 1
    ms = [(2 * i - tj) / 2 for i in range(d)]
    jz = np.diag(ms)
    jp = np.zeros((d, d))
    j = tj / 2
    for i in range(d - 1):
        m = ms[i]
        jp[i + 1, i] = math.sqrt(j * (j + 1) - m * (m + 1))
    return jz, jp, jp.T


def test_cg_equivariance():
    """X^{ab}_c intertwines: (J_a (x) 1 + 1 (x) J_b) X = X J_c for J in {J_z, J_+, J_-}."""
    for tj1, tj2 in itertools.product(spins(5), spins(5)):
        for tJ in range(abs(tj1 - tj2), tj1 + tj2 + 1, 2):
            x = su2.cg_tensor(tj1, tj2, tJ)
            for ja, jb, jc in zip(_jmats(tj1), _jmats(tj2), _jmats(tJ)):
                lhs = np.einsum("ax,xbm->abm", ja, x) + np.einsum("by,aym->abm", jb, x)
                rhs = np.einsum("abn,nm->abm", x, jc)
                assert np.allclose(lhs, rhs, atol=1e-13)


def test_z_frobenius_schur():
    """Z_a^T = chi_a Z_abar with chi_j = (-1)^(2j) (Sec. 4.2 and Sec. 5.4)."""
    for tj in spins():
        z = su2.zmat(tj)
        assert np.array_equal(z.T, (-1) ** tj * z)
        assert np.allclose(z @ z.T, np.eye(tj + 1))


# ------------------------------------------------------------------ 6j / F
def _adm_f(maxtj):
    for ta, tb, tc, td in itertools.product(spins(maxtj), repeat=4):
        for te in range(abs(ta - tb), ta + tb + 1, 2):
            if not su2.triangle(te, tc, td):
                continue
            for tf in range(abs(tb - tc), tb + tc + 1, 2):
                if su2.triangle(ta, tf, td):
                    yield ta, tb, tc, td, te, tf


def test_sixj_special_case():
    """{a b c; 0 c b} = (-1)^(a+b+c) / sqrt((2b+1)(2c+1))  (textbook)."""
    for ta, tb, tc in itertools.product(spins(), repeat=3):
        if not su2.triangle(ta, tb, tc):
            continue
        sgn, sq = su2.sixj_exact(ta, tb, tc, 0, tc, tb)
        val = sgn * math.sqrt(sq)
        assert val == pytest.approx((-1) ** ((ta + tb + tc) // 2) / math.sqrt((tb + 1) * (tc + 1)),
                                    abs=1e-15)


def test_fsymbol_racah_equals_cg_projection():
    """eq. SU2FSymbol (Racah 6j) == projection of explicit CG trees (Sec. 5.4)."""
    n = 0
    for args in _adm_f(6):
        a = su2.fsymbol_exact(*args)
        b = su2.fsymbol_from_cg(*args)
        assert abs(a - b) <= 8e-16 * max(1.0, abs(a)), args
        n += 1
    assert n > 1000


def test_fsymbol_unitary():
    for ta, tb, tc, td in itertools.product(spins(6), repeat=4):
        es = [e for e in range(abs(ta - tb), ta + tb + 1, 2) if su2.triangle(e, tc, td)]
        fs = [f for f in range(abs(tb - tc), tb + tc + 1, 2) if su2.triangle(ta, f, td)]
        if not es:
            assert not fs
            continue
        m = np.array([[su2.fsymbol_exact(ta, tb, tc, td, e, f) for f in fs] for e in es])
        assert m.shape[0] == m.shape[1]
        assert np.allclose(m @ m.T, np.eye(len(es)), atol=1e-14)


def test_fsymbol_dimension_and_fs_indicator():
    """1/d_a = |F^{a abar a}_a[I; I]|, chi_a = sign of it (Sec. 5.2, duality)."""
    for ta in spins():
        f = su2.fsymbol_exact(ta, ta, ta, ta, 0, 0)
        assert abs(f) == pytest.approx(1 / (ta + 1), abs=1e-16)
        assert math.copysign(1, f) == (-1) ** ta


def test_fsymbol_triangle():
    """Triangle equations with the unit (Sec. 5.2): F^{Iab}_c, F^{aIb}_c, F^{abI}_c are 1."""
    for ta, tb in itertools.product(spins(), repeat=2):
        for tc in range(abs(ta - tb), ta + tb + 1, 2):
            assert su2.fsymbol_exact(0, ta, tb, tc, ta, tc) == 1.0
            assert su2.fsymbol_exact(ta, 0, tb, tc, ta, tb) == 1.0
            assert su2.fsymbol_exact(ta, tb, 0, tc, tc, tb) == 1.0


# ------------------------------------------------------------------ generic pentagon / hexagon
class _Cat:
    """Multiplicity-free category from fusion rules, F and R (tables of explicit values)."""

    def __init__(self, labels, fuse, fvals, rvals):
        self.labels, self.fuse, self.fvals, self.rvals = labels, fuse, fvals, rvals

    def n(self, a, b, c):
        return c in self.fuse(a, b)

    def F(self, a, b, c, d, e, f):
        if not (self.n(a, b, e) and self.n(e, c, d) and self.n(b, c, f) and self.n(a, f, d)):
            return 0.0
        return self.fvals.get((a, b, c, d, e, f), 1.0)

    def R(self, a, b, c):
        if not self.n(a, b, c):
            return 0.0
        return self.rvals.get((a, b, c), 1.0)


def pentagon_violation(cat, ext=None):
    """max | F^{fcd}_e[g,h] F^{abh}_e[f,i] - sum_j F^{abc}_g[f,j] F^{ajd}_e[g,i] F^{bcd}_i[j,h] |
    (eq. pentagon, multiplicity-free), over external labels ``ext`` and every admissible
    internal label (enumerated through the fusion rules)."""
    fz = cat.fuse
    worst = 0.0
    for a, b, c, d in itertools.product(ext or cat.labels, repeat=4):
        for f in fz(a, b):
            for g in fz(f, c):
                for e in fz(g, d):
                    for h in fz(c, d):
                        for i in fz(b, h):
                            if e not in fz(a, i):
                                continue
                            lhs = cat.F(f, c, d, e, g, h) * cat.F(a, b, h, e, f, i)
                            rhs = sum(cat.F(a, b, c, g, f, j) * cat.F(a, j, d, e, g, i)
                                      * cat.F(b, c, d, i, j, h) for j in fz(b, c))
                            worst = max(worst, abs(lhs - rhs))
    return worst


def hexagon_violation(cat, inverse=False, ext=None):
    """max | R^{ca}_e F^{acb}_d[e,g] R^{cb}_g - sum_f F^{cab}_d[e,f] R^{cf}_d F^{abc}_d[f,g] |
    (the hexagon of Sec. 5.2 in its standard multiplicity-free form); inverse=True uses R^{-1}."""
    fz = cat.fuse
    R = (lambda a, b, c: np.conj(cat.R(a, b, c))) if inverse else cat.R
    worst = 0.0
    for a, b, c in itertools.product(ext or cat.labels, repeat=3):
        for e in fz(a, c):
            for g in fz(c, b):
                for d in fz(e, b):
                    if d not in fz(a, g):
                        continue
                    lhs = R(c, a, e) * cat.F(a, c, b, d, e, g) * R(c, b, g)
                    rhs = sum(cat.F(c, a, b, d, e, f) * R(c, f, d) * cat.F(a, b, c, d, f, g)
                              for f in fz(a, b))
                    worst = max(worst, abs(lhs - rhs))
    return worst


def _printed_category(name):
    fv, rv = {}, {}
    for ln in lines("anyon_data.txt"):
        toks = ln.split()
        if toks[0] != name:
            continue
        if toks[1] == "F":
            key = tuple(int(t) for t in toks[2:8])
            fv[key] = value(toks[8])
        else:
            key = tuple(int(t) for t in toks[2:5])
            rv[key] = cmath.exp(1j * math.pi * value(toks[6]))
    if name == "Fib":
        fuse = lambda a, b: {0: [b], 1: [a] if b == 0 else [0, 1]}[a]
        labels = [0, 1]
    else:
        table = {(0, 0): [0], (0, 1): [1], (0, 2): [2], (1, 0): [1], (1, 1): [0, 2], (1, 2): [1],
                 (2, 0): [2], (2, 1): [1], (2, 2): [0]}
        fuse = lambda a, b: table[(a, b)]
        labels = [0, 1, 2]
    return _Cat(labels, fuse, fv, rv)


@pytest.mark.parametrize("name", ["Fib", "Ising"])
def test_checkers_accept_printed_anyon_data(name):
    cat = _printed_category(name)
    assert pentagon_violation(cat) < 1e-12
    assert hexagon_violation(cat) < 1e-12
    assert hexagon_violation(cat, inverse=True) < 1e-12


def test_checkers_reject_broken_data():
    """A single flipped sign in the printed Fibonacci F must be caught by the pentagon checker."""
    cat = _printed_category("Fib")
    cat.fvals[(1, 1, 1, 1, 1, 1)] = 1 / ((1 + math.sqrt(5)) / 2)
    assert pentagon_violation(cat) > 1e-3


class _SU2Cat(_Cat):
    def __init__(self, maxtj, rsign):
        self.labels = list(spins(maxtj))
        self.fuse = lambda a, b: list(range(abs(a - b), a + b + 1, 2))
        self.rsign = rsign

    def F(self, a, b, c, d, e, f):
        return su2.fsymbol_exact(a, b, c, d, e, f)

    def R(self, a, b, c):
        if not su2.triangle(a, b, c):
            return 0.0
        return self.rsign(a, b, c)


def _r_minus(a, b, c):
    return (-1) ** ((a + b - c) // 2)


def test_su2_pentagon():
    cat = _SU2Cat(4, _r_minus)
    assert pentagon_violation(cat, ext=list(spins(4))) < 1e-13


def test_su2_rsymbol_from_cg_and_hexagon():
    """R^{ab}_c from the plain swap of CG tensors is (-1)^(a+b-c) (reading of eq. SU2RSymbol);
    it satisfies the hexagon and the unit axiom R^{Ia}_a = 1, while the printed
    (-1)^(a+b+c) gives R^{0, 1/2}_{1/2} = -1."""
    for ta, tb in itertools.product(spins(6), repeat=2):
        for tc in range(abs(ta - tb), ta + tb + 1, 2):
            assert su2.rsymbol_from_cg(ta, tb, tc) == pytest.approx(_r_minus(ta, tb, tc), abs=1e-14)
    cat = _SU2Cat(6, _r_minus)
    assert hexagon_violation(cat, ext=list(spins(6))) < 1e-13
    printed = lambda a, b, c: (-1) ** ((a + b + c) // 2)
    assert printed(0, 1, 1) == -1 and _r_minus(0, 1, 1) == 1


def test_su2_dimension_representation():
    """d_a d_b = sum_c N_ab^c d_c (eq. fusiondimrep)."""
    for ta, tb in itertools.product(spins(), repeat=2):
        assert (ta + 1) * (tb + 1) == sum(tc + 1 for tc in range(abs(ta - tb), ta + tb + 1, 2))
