"""Seeded synthetic workloads shaped like the paper's DMRG benchmarks (Sec. 6).

This module only defines inputs: graded spaces (sector -> multiplicity), which legs each
contraction pairs, the fixed XXZ matrix-product operator, and seeded N(0,1) values.  It holds no
arithmetic of the method and imports nothing from the rest of the package, so the CPU oracle's
tests and the CUDA path draw identical inputs from it.

Spaces follow the paper's benchmark shapes (Sec. 6): x : V (x) P <- V (x) P*,
W : W (x) P <- P (x) W, L : V <- V (x) W, R : W (x) V* <- V*.  Multiplicity laws stand in for the
MPSKit-derived spaces of the paper's benchmark repository (not available): U(1) charges
q = -16..16 with n_q proportional to exp(-q^2/72); SU(2) spins j = 0..4 with n_j proportional to
exp(-j^2/4); U(1) x SU(2) charge x spin pairs (Hubbard-like, see u1su2_virtual); rounded to the
stated total by largest remainder (ties: smaller |label| first).
"""

import math

import numpy as np

# ---------------------------------------------------------------------------- multiplicities


def apportion(total: int, labels, weights):
    """Largest-remainder rounding of total * w / sum(w), every share >= 1 (if total is smaller
    than the number of labels, the heaviest `total` labels get one each)."""
    labels, weights = list(labels), np.asarray(weights, dtype=np.float64)
    if total < len(labels):  # too small for every label: keep the heaviest ones, one each
        keep = sorted(range(len(labels)), key=lambda i: (-weights[i], abs(labels[i]), labels[i]))[:total]
        return {int(labels[i]): 1 for i in sorted(keep)}
    quota = total * weights / weights.sum()
    base = np.maximum(np.floor(quota).astype(np.int64), 1)
    rem = quota - np.floor(quota)
    left = total - int(base.sum())
    order = sorted(range(len(labels)), key=lambda i: (-rem[i], abs(labels[i]), labels[i]))
    i = 0
    while left > 0:
        base[order[i % len(order)]] += 1
        left -= 1
        i += 1
    while left < 0:  # only when the floor-1 constraint overshoots: take from the largest shares
        j = int(np.argmax(base))
        base[j] -= 1
        left += 1
    return {int(l): int(n) for l, n in zip(labels, base)}


def u1_virtual(D: int = 1024):
    qs = list(range(-16, 17))
    return apportion(D, qs, [math.exp(-q * q / 72.0) for q in qs])


def su2_virtual(total: int = 256):
    tjs = list(range(0, 9))  # 2j = 0..8, j = 0..4
    return apportion(total, tjs, [math.exp(-(tj / 2.0) ** 2 / 4.0) for tj in tjs])


def pair_label(a1: int, a2: int, u1_second: bool = False) -> int:
    """Integer label of the sector pair (a1, a2) of a Deligne-product symmetry: a1 * 4096 + a2,
    with a2 offset by 2048 when the second factor is U(1) (the label layout of the C ABI)."""
    return int(a1) * 4096 + int(a2) + (2048 if u1_second else 0)


def u1su2_virtual(total: int = 1024):
    """Charge x spin virtual space (Hubbard-like): q = -4..4 (particle number relative to half
    filling), 2j = 0..6 with q + 2j even, n proportional to exp(-q^2/8 - j^2/4)."""
    pairs = [(q, tj) for q in range(-4, 5) for tj in range(0, 7) if (q + tj) % 2 == 0]
    labels = [pair_label(q, tj) for q, tj in pairs]
    return apportion(total, labels, [math.exp(-q * q / 8.0 - (tj / 2.0) ** 2 / 4.0) for q, tj in pairs])


# Hubbard site: empty (q = -1, j = 0), singly occupied (q = 0, j = 1/2), doubly occupied (q = 1,
# j = 0); MPO bond: two identity channels and the hopping operators c^dagger (q = 1, j = 1/2) and
# c (q = -1, j = 1/2).  The MPO's reduced blocks are random (the fermionic signs of a true
# Hubbard MPO need fermionic braiding, which this path leaves out).
U1SU2_PHYS = {pair_label(-1, 0): 1, pair_label(0, 1): 1, pair_label(1, 0): 1}
U1SU2_MPO = {pair_label(0, 0): 2, pair_label(1, 1): 1, pair_label(-1, 1): 1}

U1_PHYS = {-1: 1, 1: 1}          # spin-1/2, charge 2 S_z
U1_MPO = {-2: 1, 0: 3, 2: 1}     # XXZ bond space
SU2_PHYS = {1: 1}                # j = 1/2
SU2_MPO = {0: 2, 2: 1}           # 2 (0) (+) (1), the Heisenberg bond of Sec. 6.1

# SU(2) Heisenberg MPO (J = 1) on W : W (x) P <- P (x) W with W = 2 (0) (+) (1), P = (1/2): its
# ten reduced entries in storage order, as written to tests/golden/heisenberg_su2_mpo.txt by
# tests/golden/make_heisenberg_su2_mpo.py (the oracle's projection of the dense lower-triangular
# MPO with identity, spin-vector and J S.S channels).
HEISENBERG_SU2_MPO = (1.0, 0.0, -0.8660254037844386, 0.0, 1.0, 0.0, 0.0, 0.8660254037844386, 0.0, 0.0)

# bond state b of the XXZ MPO -> (charge, outer index); states 0 (identity before), 3 (S_z),
# 4 (identity after) share charge 0; 1 carries S+, 2 carries S-.
_BOND = {0: (0, 0), 1: (-2, 0), 2: (2, 0), 3: (0, 1), 4: (0, 2)}


def xxz_mpo_entries(jz: float = 1.0, jxy: float = 1.0):
    """Non-zero entries of W[(w_l, s'), (s, w_r)] = <s'| W[w_l][w_r] |s> for the lower-triangular
    XXZ MPO {I; S+; S-; Sz; (Jxy/2) S-, (Jxy/2) S+, Jz Sz, I}.

    Returns [((w_l charge, w_l outer), s' charge, s charge, (w_r charge, w_r outer), value)],
    physical charges 2 S_z = +-1.
    """
    ops = {
        "I": {(1, 1): 1.0, (-1, -1): 1.0},
        "S+": {(1, -1): 1.0},
        "S-": {(-1, 1): 1.0},
        "Sz": {(1, 1): 0.5, (-1, -1): -0.5},
    }
    table = [(0, 0, "I", 1.0), (1, 0, "S+", 1.0), (2, 0, "S-", 1.0), (3, 0, "Sz", 1.0),
             (4, 1, "S-", jxy / 2), (4, 2, "S+", jxy / 2), (4, 3, "Sz", jz), (4, 4, "I", 1.0)]
    out = []
    for wl, wr, name, scale in table:
        for (sp, s), v in ops[name].items():
            out.append((_BOND[wl], sp, s, _BOND[wr], scale * v))
    return out


# ---------------------------------------------------------------------------- random values


def normal(seed: int, n: int) -> np.ndarray:
    """n iid N(0,1) doubles from numpy PCG64 with the given seed."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(n)


def normal_complex(seed: int, n: int) -> np.ndarray:
    """n complex values with iid N(0, 1/2) real and imaginary parts."""
    g = np.random.Generator(np.random.PCG64(seed))
    return (g.standard_normal(n) + 1j * g.standard_normal(n)) * math.sqrt(0.5)


def integer_valued(seed: int, n: int, bound: int = 255) -> np.ndarray:
    """n integers in [-bound, bound] as doubles (exactness checks of split-precision GEMMs)."""
    g = np.random.Generator(np.random.PCG64(seed))
    return g.integers(-bound, bound + 1, n).astype(np.float64)


# ---------------------------------------------------------------------------- contractions
# A contraction spec is (pA, qA, pB, qB, pAB, qAB) in the 0-based leg numbering of Algorithm 4.

# C[a,b,e,f] = sum_{c,d} A[a,c,b,d] B[d,c,e,f]; A : V (x) V <- V (x) V, B : V (x) V* <- V (x) V
# (B's second codomain leg is dual so that the contracted pair is well typed).
C0_SPEC = ((0, 2), (3, 1), (0, 1), (2, 3), (0, 1), (2, 3))

# Two-site effective Hamiltonian x' = L . x . W . W . R as four pairwise contractions.
#   T1 = L x   : L[a'; a, w1] x[a, s1; b, s2]
#   T2 = T1 W  : contract w1 and s1 with W[w_l, s'; s, w_r]
#   T3 = T2 W  : contract w2 and s2
#   x' = T3 R  : contract w3 and b with R[w3, b'; b]; result has the structure of x
HEFF_SPECS = [
    ((0, 2), (1,), (0,), (1, 2, 3), (0, 1), (2, 3, 4)),
    ((0, 3, 4), (1, 2), (0, 2), (1, 3), (0, 1, 2), (3, 4)),
    ((0, 1, 3), (4, 2), (0, 2), (1, 3), (0, 1, 2), (3, 4)),
    ((0, 2, 3), (4, 1), (0, 2), (1,), (0, 1), (3, 2)),
]

# Environment applied to the two-site tensor: T = L x (the first step of the chain).
LX_SPEC = HEFF_SPECS[0]

# Single-site effective Hamiltonian (Algorithm 11): x' = ((L x) W) R with x : V (x) P <- V.
# Steps: T1 = L x over the left virtual leg; T2 = T1 W over (MPO bond, physical leg);
# x' = T2 R over (MPO bond, right virtual leg); x' has the structure of x.
HEFF1_SPECS = [
    ((0, 2), (1,), (0,), (1, 2), (0, 1), (2, 3)),
    ((0, 3), (1, 2), (0, 2), (1, 3), (0, 1), (2, 3)),
    ((0, 2), (3, 1), (0, 2), (1,), (0, 1), (2,)),
]


def heff_spaces(sym: str, D: int):
    """(V, P, W) sector dicts of the two-site heff workload."""
    if sym == "U1":
        return u1_virtual(D), U1_PHYS, U1_MPO
    if sym == "U1xSU2":
        return u1su2_virtual(D), U1SU2_PHYS, U1SU2_MPO
    return su2_virtual(D), SU2_PHYS, SU2_MPO


def heff_legs(V, P, W):
    """Leg lists ((codomain), (domain)) of x, L, W, R as (sectors, dual) pairs."""
    x = ([(V, False), (P, False)], [(V, False), (P, True)])
    L = ([(V, False)], [(V, False), (W, False)])
    Wt = ([(W, False), (P, False)], [(P, False), (W, False)])
    R = ([(W, False), (V, True)], [(V, True)])
    return {"x": x, "L": L, "W": Wt, "R": R}


def heff1_legs(V, P, W):
    """Leg lists of the single-site workload: x : V (x) P <- V; L, W, R as in heff_legs."""
    legs = heff_legs(V, P, W)
    legs["x"] = ([(V, False), (P, False)], [(V, False)])
    return legs


CONFIGS = {
    "c0_u1_small": dict(sym="U1", D=9, kind="c0"),
    "c1_u1_heff_d1024": dict(sym="U1", D=1024, kind="heff"),
    "c2a_su2_lx_n256": dict(sym="SU2", D=256, kind="lx"),
    "c2b_su2_lx_n512": dict(sym="SU2", D=512, kind="lx"),
    "c3_u1_heff_d4096": dict(sym="U1", D=4096, kind="heff"),
    "c5_u1_heff1_d4096": dict(sym="U1", D=4096, kind="heff1"),
    "c5_su2_heff1_n1024": dict(sym="SU2", D=1024, kind="heff1"),
    "c3_su2_lx_n1024": dict(sym="SU2", D=1024, kind="lx"),
    "c6_u1su2_heff_n2048": dict(sym="U1xSU2", D=2048, kind="heff"),
    "c7_su2_heisenberg_heff_n1024": dict(sym="SU2", D=1024, kind="heff", mpo="heisenberg"),
}
