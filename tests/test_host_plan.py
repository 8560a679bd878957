"""Host logic of libtk against the oracle (no GPU): structures, exact symbols, permute transforms.

The library side computes recoupling coefficients with F/B/R moves and Racah 6j symbols; the
oracle projects permuted explicit CG trees.  The two share no code.
"""

import itertools
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle import SU2, U1, Z2, GradedSpace, TensorStructure
from oracle.symmetry import U1xSU2, Z2xU1
from oracle import ops, su2
from paper_2508_10076_gb300 import api, build_library
from paper_2508_10076_gb300._abi import SIGNATURES


@pytest.fixture(scope="module")
def hctx():
    build_library()
    return api.Context(-1)


def test_library_exports_every_declared_symbol():
    build_library()
    import ctypes
    from paper_2508_10076_gb300.build import LIB
    lib = ctypes.CDLL(LIB)
    with open(f"{ROOT}/include/tk.h") as fh:
        header = fh.read()
    declared = set(re.findall(r"\b(tk_[a-z0-9_]+)\s*\(", header))
    assert declared == set(SIGNATURES), declared ^ set(SIGNATURES)
    for name in declared:
        assert hasattr(lib, name), name


def _mk(ctx, sym, spec):
    cod, dom = spec
    o_cod = [GradedSpace(sym, s, d) for s, d in cod]
    o_dom = [GradedSpace(sym, s, d) for s, d in dom]
    l_cod = [ctx.space(sym.name, s, d) for s, d in cod]
    l_dom = [ctx.space(sym.name, s, d) for s, d in dom]
    return TensorStructure(o_cod, o_dom), ctx.tmap(l_cod, l_dom)


def _same_structure(ost, lt):
    assert lt.numel == ost.numel
    assert lt.blocks() == [(c, r, k, off) for c, r, k, off in ost.blocks]
    lib_pairs = lt.treepairs()
    assert len(lib_pairs) == len(ost.pairs)
    for (unc, si, c, fi, off, ld, dims), p in zip(lib_pairs, ost.pairs):
        assert unc == p.split_unc + p.fuse_unc
        assert si == p.split_inner and fi == p.fuse_inner and c == p.coupled
        assert (off, ld, dims) == (p.offset, p.ld, p.dims)


_P, _Q = U1xSU2.pair, Z2xU1.pair

SPECS = [
    (SU2, ([({0: 1, 1: 1}, False)] * 2, [({0: 1, 1: 1}, False)] * 2)),
    (SU2, ([({0: 2, 1: 1, 2: 2}, False), ({1: 1}, False)], [({0: 1, 1: 2, 2: 1}, True), ({1: 1}, True)])),
    (SU2, ([({1: 2, 3: 1}, True), ({0: 1, 2: 1}, False), ({1: 1}, False)], [({0: 1, 2: 2}, False)])),
    (SU2, ([({0: 1, 2: 1}, True)], [({1: 1, 3: 1}, False), ({1: 2}, True), ({0: 1, 2: 1, 4: 1}, False)])),
    (SU2, ([], [({1: 1, 3: 1}, False), ({1: 2, 2: 1}, True), ({0: 1, 1: 1}, False)])),
    (U1, ([({-2: 1, -1: 2, 0: 3, 1: 2, 2: 1}, False)] * 2, [({-2: 1, -1: 2, 0: 3, 1: 2, 2: 1}, False)] * 2)),
    (U1, ([({-1: 2, 1: 1}, True), ({0: 1, 2: 2}, False)], [({-1: 1, 1: 3, 3: 1}, False), ({1: 1, -1: 1}, True)])),
    (Z2, ([({0: 2, 1: 1}, False), ({0: 1, 1: 2}, True), ({1: 1}, False)], [({0: 3, 1: 1}, False)])),
    # Deligne products: charge x spin (non-abelian) and parity x charge (abelian)
    (U1xSU2, ([({_P(-1, 1): 1, _P(0, 0): 2, _P(1, 1): 1}, False), ({_P(1, 1): 1, _P(-1, 1): 1}, False)],
              [({_P(0, 0): 1, _P(0, 2): 1, _P(1, 1): 1, _P(-1, 1): 1}, True), ({_P(1, 1): 1}, True)])),
    (U1xSU2, ([({_P(0, 1): 2, _P(1, 0): 1}, True), ({_P(0, 1): 1, _P(1, 2): 1}, False), ({_P(-1, 1): 1}, False)],
              [({_P(0, 0): 1, _P(0, 2): 1, _P(1, 1): 1}, False)])),
    (Z2xU1, ([({_Q(0, -1): 1, _Q(1, 0): 2, _Q(0, 1): 1}, False), ({_Q(1, 1): 1, _Q(0, -1): 1}, True)],
             [({_Q(1, 0): 1, _Q(0, 0): 2, _Q(1, 2): 1}, False), ({_Q(0, 1): 1}, True)])),
]


@pytest.mark.parametrize("k", range(len(SPECS)))
def test_structure_bit_exact(hctx, k):
    sym, spec = SPECS[k]
    ost, lt = _mk(hctx, sym, spec)
    _same_structure(ost, lt)


def _oracle_transform_offsets(ost, p, q):
    out, tr = ops.permute_transform(ost, p, q)
    idx_in = ost.pair_index()
    idx_out = out.pair_index()
    res = {}
    for src, lst in tr.items():
        for dst, coef in lst:
            res[(idx_in[src].offset, idx_out[dst].offset)] = coef
    return out, res


@pytest.mark.parametrize("k", range(len(SPECS)))
def test_permute_transform_matches_oracle(hctx, k):
    """F/B/R-move coefficients (library) == overlap-route coefficients (oracle), all (p, q) tried
    for rank <= 3 and a random sample for rank 4."""
    sym, spec = SPECS[k]
    ost, lt = _mk(hctx, sym, spec)
    n = ost.nleg
    perms = list(itertools.permutations(range(n)))
    rng = np.random.default_rng(k)
    if len(perms) > 12:
        perms = [perms[i] for i in rng.choice(len(perms), 12, replace=False)]
    for perm in perms:
        for split in range(n + 1):
            p, q = tuple(perm[:split]), tuple(perm[split:])
            out, ref = _oracle_transform_offsets(ost, p, q)
            plan = api.permute_plan(hctx, lt, p, q)
            _same_structure(out, plan.output())
            got = plan.transform(0)
            if got is None:  # identity permute
                assert p == tuple(range(len(ost.cod))) and q == tuple(range(len(ost.cod), n))
                continue
            gd = {(s, d): c for s, d, c in got}
            keys = set(gd) | set(ref)
            for key in keys:
                assert abs(gd.get(key, 0.0) - ref.get(key, 0.0)) < 1e-12, (p, q, key)


def test_fsymbols_bit_exact(hctx):
    """Library F-symbols (C++ big integers) == oracle F-symbols (Python fractions), bit for bit."""
    n = 0
    for ta, tb, tc, td in itertools.product(range(0, 7), repeat=4):
        for te in range(abs(ta - tb), ta + tb + 1, 2):
            for tf in range(abs(tb - tc), tb + tc + 1, 2):
                ref = su2.fsymbol_exact(ta, tb, tc, td, te, tf)
                got = api.fsymbol("SU2", ta, tb, tc, td, te, tf)
                assert got == ref, (ta, tb, tc, td, te, tf, got, ref)
                n += 1
    assert n > 10000
    for ta, tb in itertools.product(range(9), repeat=2):
        for tc in range(abs(ta - tb), ta + tb + 1, 2):
            assert api.rsymbol("SU2", ta, tb, tc) == su2.rsymbol_from_cg(ta, tb, tc) or \
                abs(api.rsymbol("SU2", ta, tb, tc) - su2.rsymbol_from_cg(ta, tb, tc)) < 1e-14


def test_contract_plan_structure_and_flops(hctx):
    """C0: A~ has square per-charge GEMMs (1,4,10,16,19,16,10,4,1), 34,362 block flops."""
    v = {-2: 1, -1: 2, 0: 3, 1: 2, 2: 1}
    V, Vd = hctx.space("U1", v), hctx.space("U1", v, True)
    A = hctx.tmap([V, V], [V, V])
    B = hctx.tmap([V, Vd], [V, V])
    plan = api.contract_plan(hctx, A, (0, 2), (3, 1), B, (0, 1), (2, 3), (0, 1), (2, 3))
    assert plan.flops == 34362
    assert plan.transform(1) is None  # B is used as is
    out = plan.output()
    oa = TensorStructure([GradedSpace(U1, v), GradedSpace(U1, v)], [GradedSpace(U1, v)] * 2)
    ob = TensorStructure([GradedSpace(U1, v), GradedSpace(U1, v, True)], [GradedSpace(U1, v)] * 2)
    xa, xb = np.zeros(oa.numel), np.zeros(ob.numel)
    cs, _ = ops.contract(oa, xa, (0, 2), (3, 1), ob, xb, (0, 1), (2, 3), (0, 1), (2, 3), tier="block")
    _same_structure(cs, out)


def test_errors_are_reported(hctx):
    V = hctx.space("SU2", {1: 1})
    t = hctx.tmap([V], [V])
    with pytest.raises(api.TKError) as e:
        api.permute_plan(hctx, t, (0, 0), ())
    assert e.value.code == 3
    W = hctx.space("SU2", {0: 1})
    t2 = hctx.tmap([W], [W])
    with pytest.raises(api.TKError) as e:
        api.contract_plan(hctx, t, (0,), (1,), t2, (0,), (1,), (0,), (1,))
    assert e.value.code == 2
    with pytest.raises(api.TKError) as e:
        hctx.space("Z2", {2: 1})
    assert e.value.code == 4


def test_adjoint_plan_structure_matches_oracle(hctx):
    """The adjoint plan's output structure is the oracle's (domain and codomain exchanged), bit
    for bit, on a host-only context."""
    from harness import ostruct
    for sym, legs in (("SU2", ([({0: 2, 1: 1}, False), ({1: 2}, True)], [({0: 1, 1: 2, 2: 1}, False)])),
                      ("U1", ([({-1: 2, 0: 3}, False)], [({0: 2, 1: 1}, True), ({-1: 1, 1: 2}, False)]))):
        ost = ostruct(sym, legs)
        cod, dom = legs
        t = hctx.tmap([hctx.space(sym, s, d) for s, d in cod], [hctx.space(sym, s, d) for s, d in dom])
        plan = api.adjoint_plan(hctx, t)
        os2, _ = ops.adjoint_block(ost, np.zeros(ost.numel))
        assert plan.output().blocks() == [(c, r, k, o) for c, r, k, o in os2.blocks]


def test_svd_plan_structures_match_oracle(hctx):
    """U : cod <- W and V^dagger : W <- dom with W = sum_c (c, min(rows_c, cols_c)), bit for bit."""
    from harness import ostruct
    for sym, legs in (("SU2", ([({0: 2, 1: 2}, False), ({1: 1}, False)], [({0: 1, 1: 2, 2: 1}, False), ({1: 1}, True)])),
                      ("U1", ([({-1: 2, 0: 3}, False), ({1: 1, -1: 1}, False)], [({0: 2, 1: 1}, False)]))):
        ost = ostruct(sym, legs)
        cod, dom = legs
        t = hctx.tmap([hctx.space(sym, s, d) for s, d in cod], [hctx.space(sym, s, d) for s, d in dom])
        plan = api.svd_plan(hctx, t)
        u, vh, n = plan.outputs()
        w = GradedSpace(ost.sym, {c: min(r, k) for c, r, k, _ in ost.blocks if min(r, k) > 0})
        ou, ov = TensorStructure(ost.cod, [w]), TensorStructure([w], ost.dom)
        assert u.blocks() == [(c, r, k, o) for c, r, k, o in ou.blocks]
        assert vh.blocks() == [(c, r, k, o) for c, r, k, o in ov.blocks]
        assert n == sum(min(r, k) for _, r, k, _ in ost.blocks)


def test_mpo_leg_permute_uses_vector_tiles(hctx):
    """An environment R : W (x) V' <- V' permuted to (W, V'_dom) <- V'_cod (the T3.R step of the
    heff chain): the MPO leg (extent 1-4 per sector) is contiguous on both sides, so every task is
    a transpose of short vectors, none element-wise."""
    legs = ([({-2: 2, 0: 3, 2: 4}, False), ({-1: 37, 0: 50, 1: 41}, True)], [({-1: 19, 0: 50, 1: 33}, True)])
    cod, dom = legs
    t = hctx.tmap([hctx.space("U1", s, d) for s, d in cod], [hctx.space("U1", s, d) for s, d in dom])
    p = api.permute_plan(hctx, t, (0, 2), (1,))
    st = p.permute_stats(0)
    assert st["generic_tasks"] == 0 and st["run_tasks"] == 0
    assert st["transpose_elems"] == t.numel
    ost = TensorStructure([GradedSpace(U1, s, d) for s, d in cod], [GradedSpace(U1, s, d) for s, d in dom])
    out, _ = _oracle_transform_offsets(ost, (0, 2), (1,))
    _same_structure(out, p.output())


def test_compose_plan_structure_matches_oracle(hctx):
    """A o B (Sec. 2.3) as a plan: output structure and block flops as the oracle's composition;
    a domain / codomain mismatch is refused."""
    v = {-1: 2, 0: 3, 1: 1}
    w = {0: 2, 1: 2}
    la = ([(v, False), (w, True)], [(v, False)])
    lb = ([(v, False)], [(w, False)])
    A, B = _mk(hctx, U1, la)[1], _mk(hctx, U1, lb)[1]
    oa, ob = _mk(hctx, U1, la)[0], _mk(hctx, U1, lb)[0]
    plan = api.compose_plan(hctx, A, B)
    cs, _ = ops.compose_block(oa, np.zeros(oa.numel), ob, np.zeros(ob.numel))
    _same_structure(cs, plan.output())
    bb = {c: cols for c, rows, cols, _ in ob.blocks}
    assert plan.flops == sum(2 * rows * k * bb[c] for c, rows, k, _ in oa.blocks if c in bb)
    with pytest.raises(api.TKError) as e:
        api.compose_plan(hctx, B, A)  # dom(B) = W is not cod(A) = V (x) W*
    assert e.value.code == 2
