"""Pins of the oracle's block layout: the paper's worked examples and brute-force counting."""

import itertools
import math

import numpy as np
import pytest

from golden_io import lines
from oracle import SU2, U1, Z2, GradedSpace, TensorStructure
from oracle.symmetry import U1xSU2, Z2xU1
from harness import total_generators
from oracle.dense import embed
from oracle.ops import permute_spaces


def _z2_channels(struct):
    """{c: (row channels, col channels)} with labels written as +/- strings."""
    sign = {0: "+", 1: "-"}
    out = {}
    for c, rows, cols, off in struct.blocks:
        prs = [p for p in struct.pairs if p.coupled == c]
        rws = []
        for p in prs:
            s = "".join(sign[a] for a in p.split_unc)
            if s not in rws:
                rws.append(s)
        cls = []
        for p in prs:
            s = "".join(sign[a] for a in p.fuse_unc)
            if s not in cls:
                cls.append(s)
        # storage order: sort by offsets
        rws.sort(key=lambda s: min(p.row_off for p in prs if "".join(sign[a] for a in p.split_unc) == s))
        cls.sort(key=lambda s: min(p.col_off for p in prs if "".join(sign[a] for a in p.fuse_unc) == s))
        out[sign[c]] = (rws, cls)
    return out


def test_z2_worked_examples():
    v = GradedSpace(Z2, {0: 1, 1: 1})
    t = TensorStructure([v, v], [v, v])
    bent_cod, bent_dom = permute_spaces(t, (0, 1, 3), (2,))
    bent = TensorStructure(bent_cod, bent_dom)
    got = {"grouped": _z2_channels(t), "bent": _z2_channels(bent)}
    n = 0
    for ln in lines("z2_examples.txt"):
        kind, c, _, rest = ln.split(None, 3)
        rows, cols = rest.split("|")
        assert got[kind][c] == (rows.split(), cols.split()), (kind, c)
        n += 1
    assert n == 4


def test_su2_worked_example_structure():
    """V = V^(0) (+) V^(1/2): five splitting trees, nine reduced elements, blocks 2x2, 2x2, 1x1,
    81 dense parameters vs 9 (Sec. 4.3, grouping and splitting indices)."""
    v = GradedSpace(SU2, {0: 1, 1: 1})
    t = TensorStructure([v, v], [v, v])
    assert [(c, r, k) for c, r, k, _ in t.blocks] == [(0, 2, 2), (1, 2, 2), (2, 1, 1)]
    assert len({(p.split_unc, p.split_inner, p.coupled) for p in t.pairs}) == 5
    assert t.numel == 9
    assert math.prod(s.dim for s in t.spaces()) == 81


def test_block_rows_count_fusion_multiplicities():
    """N_c^W = sum_{a,b} N_a N_b N_ab^c  (Sec. 4.1, grouping isomorphism)."""
    v = GradedSpace(SU2, {0: 2, 1: 3, 2: 1, 3: 2})
    w = GradedSpace(SU2, {1: 1, 2: 2}, dual=True)
    t = TensorStructure([v, w], [GradedSpace(SU2, {c: 1 for c in range(0, 6)})])
    for c, rows, cols, off in t.blocks:
        expect = sum(na * nb for a, na in v.sectors.items() for b, nb in w.sectors.items()
                     if abs(a - b) <= c <= a + b and (a + b + c) % 2 == 0)
        assert rows == expect


# ------------------------------------------------------------------ brute force invariants
_P, _Q = U1xSU2.pair, Z2xU1.pair

CASES = [
    (SU2, [({0: 1, 1: 1}, False), ({0: 1, 1: 1}, False)], [({0: 1, 1: 1}, False), ({0: 1, 1: 1}, False)]),
    (SU2, [({1: 2, 2: 1}, False), ({1: 1}, True)], [({0: 1, 2: 1}, False), ({1: 1, 3: 1}, True)]),
    (SU2, [({0: 1, 1: 1, 2: 1}, True)], [({1: 1}, False), ({0: 2, 2: 1}, False), ({1: 1}, True)]),
    (U1, [({-1: 1, 0: 2, 1: 1}, False), ({-1: 1, 1: 2}, True)], [({0: 1, 2: 1, -2: 1}, False)]),
    (Z2, [({0: 2, 1: 1}, False), ({0: 1, 1: 1}, True)], [({0: 1, 1: 2}, True), ({1: 1}, False)]),
    (U1xSU2, [({_P(0, 0): 1, _P(1, 1): 1}, False), ({_P(-1, 1): 1, _P(1, 1): 1}, True)],
     [({_P(0, 0): 1, _P(0, 2): 1, _P(2, 0): 1}, False)]),
    (Z2xU1, [({_Q(0, 0): 1, _Q(1, 1): 2}, False), ({_Q(1, -1): 1, _Q(0, 1): 1}, True)],
     [({_Q(1, 0): 1, _Q(0, 2): 1, _Q(1, 2): 1}, True)]),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_numel_equals_invariant_subspace_dimension(case):
    """Brute force: the number of reduced coefficients equals dim of the invariant subspace, and
    the dense embedding maps onto it (Schur's lemma / Wigner-Eckart, Sec. 3.1 and 4.1)."""
    sym, cod, dom = CASES[case]
    st = TensorStructure([GradedSpace(sym, s, d) for s, d in cod], [GradedSpace(sym, s, d) for s, d in dom])
    gens = np.concatenate(total_generators(st), axis=0)
    sv = np.linalg.svd(gens, compute_uv=False)
    n = math.prod(sp.dim for sp in st.spaces())
    null_dim = n - int(np.sum(sv > 1e-9))
    assert st.numel == null_dim
    # embedding of each unit reduced vector: invariant, and orthogonal with norm^2 = d_c
    basis = np.stack([embed(st, np.eye(st.numel)[i]).reshape(-1) for i in range(st.numel)])
    assert np.abs(gens @ basis.T).max() < 1e-12
    gram = basis @ basis.T
    dc = np.array([sym.dim(p.coupled) for p in sorted(st.pairs, key=lambda p: p.offset)
                   for _ in range(math.prod(p.dims))])
    # reorder dc by flat position
    diag = np.zeros(st.numel)
    for p in st.pairs:
        n1 = len(st.cod)
        r = math.prod(p.dims[:n1]); c = math.prod(p.dims[n1:])
        for j in range(c):
            diag[p.offset + j * p.ld: p.offset + j * p.ld + r] = sym.dim(p.coupled)
    assert np.allclose(gram, np.diag(diag), atol=1e-12)
    del dc


def test_u1_charge_conservation_zeros():
    """Dense U(1) tensors vanish wherever codomain charge != domain charge (eq. abeliantensorzeros)."""
    v = GradedSpace(U1, {-1: 1, 0: 2, 1: 1})
    st = TensorStructure([v, v], [v.flip()])
    x = np.random.default_rng(1).standard_normal(st.numel)
    d = embed(st, x)
    ch = [a for a, n in v.sectors.items() for _ in range(n)]
    for i, j, k in itertools.product(range(v.dim), repeat=3):
        total = ch[i] + ch[j] - (-ch[k])   # domain leg V* carries charge -q "as if normal"
        if total != 0:
            assert d[i, j, k] == 0.0
