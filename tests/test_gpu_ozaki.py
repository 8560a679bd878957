"""Split-precision (Ozaki BF16 on tcgen05) sector GEMMs against FP64 and the oracle."""

import numpy as np
import pytest

from harness import oracle_heff, oracle_heff_inputs, ostruct, rel_frobenius_per_block
from oracle import ops
from paper_2508_10076_gb300 import build_library
from paper_2508_10076_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPLIT_TOL = 1e-10


@pytest.fixture(scope="module")
def gctx():
    assert torch.cuda.is_available()
    build_library()
    from paper_2508_10076_gb300 import api
    ctx = api.Context(0)
    yield ctx
    ctx.sync()


def _api():
    from paper_2508_10076_gb300 import api
    return api


def _tm(ctx, sym, legs):
    cod, dom = legs
    return ctx.tmap([ctx.space(sym, s, d) for s, d in cod], [ctx.space(sym, s, d) for s, d in dom])


def _run(ctx, plan, a, b):
    api = _api()
    c = torch.full((plan.output().numel,), float("nan"), dtype=torch.float64, device="cuda")
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    api.contract(ctx, plan, a, b, c, ws)
    ctx.sync()
    return c


def test_integer_inputs_are_exact(gctx):
    """Integer entries |x| <= 255: every slice product and every exact level is an integer times a
    power of two, so the split-precision result equals the FP64 result bit for bit (this also
    checks that tensor-core FP32 accumulation adds these values without rounding)."""
    api = _api()
    legs_a = ([({-1: 40, 0: 150, 1: 60}, False), ({0: 2, 1: 1}, False)], [({-1: 30, 0: 200, 1: 45}, False)])
    legs_b = ([({-1: 30, 0: 200, 1: 45}, False)], [({-1: 50, 0: 170, 1: 20}, False)])
    A, B = _tm(gctx, "U1", legs_a), _tm(gctx, "U1", legs_b)
    xa = torch.from_numpy(wl.integer_valued(1, A.numel)).cuda()
    xb = torch.from_numpy(wl.integer_valued(2, B.numel)).cuda()
    spec = ((0, 1), (2,), (0,), (1,), (0, 1), (2,))
    p64 = api.contract_plan(gctx, A, *spec[:2], B, *spec[2:])
    poz = api.contract_plan(gctx, A, *spec[:2], B, *spec[2:], gemm="ozaki")
    c64, coz = _run(gctx, p64, xa, xb), _run(gctx, poz, xa, xb)
    assert torch.equal(c64, coz)


@pytest.mark.parametrize("slices,tol", [(6, SPLIT_TOL), (7, 1e-12)])
def test_c0_split_precision(gctx, slices, tol):
    api = _api()
    v = {-2: 1, -1: 2, 0: 3, 1: 2, 2: 1}
    la = ([(v, False), (v, False)], [(v, False), (v, False)])
    lb = ([(v, False), (v, True)], [(v, False), (v, False)])
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    xa, xb = wl.normal(0, oa.numel), wl.normal(1, ob.numel)
    cs, ref = ops.contract(oa, xa, *wl.C0_SPEC[:2], ob, xb, *wl.C0_SPEC[2:], tier="dense")
    A, B = _tm(gctx, "U1", la), _tm(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, *wl.C0_SPEC[:2], B, *wl.C0_SPEC[2:], gemm="ozaki", slices=slices)
    c = _run(gctx, plan, torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda())
    assert rel_frobenius_per_block(cs, c.cpu().numpy(), ref) <= tol


def test_heff_chain_split_precision_d1024(gctx):
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(gctx, "U1", 1024, gemm="ozaki")
    ref = oracle_heff("U1", 1024, tier="block")
    t = ch.steps[0].run(ch.dev["L"], ch.dev["x"])
    outs = [t]
    for i, other in ((1, "W"), (2, "W"), (3, "R")):
        t = ch.steps[i].run(t, ch.dev[other])
        outs.append(t)
    gctx.sync()
    for i, ((cs, rd), b) in enumerate(zip(ref, outs)):
        err = rel_frobenius_per_block(cs, b.cpu().numpy(), rd)
        assert err <= SPLIT_TOL, (i, err)


def test_su2_lx_split_precision(gctx):
    from paper_2508_10076_gb300.chain import LxContraction
    lx = LxContraction(gctx, "SU2", 256, gemm="ozaki")
    got = lx.run()
    gctx.sync()
    st, data = oracle_heff_inputs("SU2", 256)
    cs, ref = ops.contract(st["L"], data["L"], *wl.LX_SPEC[:2], st["x"], data["x"], *wl.LX_SPEC[2:], tier="block")
    assert rel_frobenius_per_block(cs, got.cpu().numpy(), ref) <= SPLIT_TOL


def test_long_inner_dimension_uses_segments(gctx):
    """K = 5000: few output tiles, so the inner dimension is split across CTAs (parts added in
    FP64 in part order), and each part still spans two exact 1024-deep segments; ragged M, N
    tails.  Repeated runs agree bit for bit."""
    api = _api()
    la = ([({0: 300, 1: 7}, False)], [({0: 5000, 1: 3}, False)])
    lb = ([({0: 5000, 1: 3}, False)], [({0: 200, 1: 5}, False)])
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    xa, xb = wl.normal(5, oa.numel), wl.normal(6, ob.numel)
    cs, ref = ops.contract(oa, xa, (0,), (1,), ob, xb, (0,), (1,), (0,), (1,), tier="block")
    A, B = _tm(gctx, "U1", la), _tm(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, (0,), (1,), B, (0,), (1,), (0,), (1,), gemm="ozaki")
    c = _run(gctx, plan, torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda())
    assert rel_frobenius_per_block(cs, c.cpu().numpy(), ref) <= SPLIT_TOL
    c2 = _run(gctx, plan, torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda())
    assert torch.equal(c, c2)


def test_scales_span_many_binades(gctx):
    """Rows and columns scaled by 2^(+-40): per-row/per-column power-of-two scales absorb them."""
    api = _api()
    la = ([({0: 130, 1: 20}, False)], [({0: 100, 1: 9}, False)])
    lb = ([({0: 100, 1: 9}, False)], [({0: 140, 1: 33}, False)])
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    rng = np.random.default_rng(9)
    xa = wl.normal(7, oa.numel) * np.exp2(rng.integers(-40, 41, oa.numel))
    xb = wl.normal(8, ob.numel) * np.exp2(rng.integers(-40, 41, ob.numel))
    cs, ref = ops.contract(oa, xa, (0,), (1,), ob, xb, (0,), (1,), (0,), (1,), tier="block")
    A, B = _tm(gctx, "U1", la), _tm(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, (0,), (1,), B, (0,), (1,), (0,), (1,), gemm="ozaki")
    c = _run(gctx, plan, torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda())
    # Per-row (per-column) scales 2^e <= 2 max|a| and 7 s fraction bits: each operand entry is off
    # by at most 2^(-7s) max|a|, two such terms per product; the dropped slice pairs (i + j = s,
    # s - 1 of them with both digits <= 64, each below 2^12 2^(-7(s+2)) 2^(e_m + f_n)) add at most
    # (s - 1) 2^(-7s) max|a| max|b| per k.  Together: below 8 2^(-7s) K max|a| max|b| for s = 6.
    got = c.cpu().numpy()
    for (ca, ra, ka, oa_), (cb, rb, kb, ob_), (cc, rc, kc, oc) in zip(oa.blocks, ob.blocks, cs.blocks):
        am = xa[oa_:oa_ + ra * ka].reshape(ka, ra).T
        bm = xb[ob_:ob_ + rb * kb].reshape(kb, rb).T
        bound = 8 * 2.0 ** (-42) * ka * np.abs(am).max(axis=1)[:, None] * np.abs(bm).max(axis=0)[None, :]
        err = np.abs(got[oc:oc + rc * kc] - ref[oc:oc + rc * kc]).reshape(kc, rc).T
        assert np.all(err <= bound)


def _elementwise_bound_check(oa, xa, ob, xb, cs, ref, got, factor):
    """|got - ref| <= factor K max|a_m.| max|b_.n| element by element (the split's error is relative
    to the row and column maxima, which the power-of-two scales follow)."""
    for (ca, ra, ka, oa_), (cb, rb, kb, ob_), (cc, rc, kc, oc) in zip(oa.blocks, ob.blocks, cs.blocks):
        am = xa[oa_:oa_ + ra * ka].reshape(ka, ra).T
        bm = xb[ob_:ob_ + rb * kb].reshape(kb, rb).T
        bound = factor * ka * np.abs(am).max(axis=1)[:, None] * np.abs(bm).max(axis=0)[None, :]
        err = np.abs(got[oc:oc + rc * kc] - ref[oc:oc + rc * kc]).reshape(kc, rc).T
        assert np.all(err <= bound)


PREP_CASES = [
    # (A legs, B legs): one k-chunk per CTA; several chunks of a deep tile per CTA (K = 5000, up
    # to eight CTAs per tile, so CTAs own two chunks in images and more straight from L2); ragged
    # rows, columns and inner dimensions throughout
    (([({0: 130, 1: 20}, False)], [({0: 100, 1: 9}, False)]),
     ([({0: 100, 1: 9}, False)], [({0: 140, 1: 33}, False)])),
    (([({0: 300, 1: 7}, False)], [({0: 5000, 1: 3}, False)]),
     ([({0: 5000, 1: 3}, False)], [({0: 200, 1: 5}, False)])),
]


@pytest.mark.parametrize("gemm,tol", [("ozaki", SPLIT_TOL), ("tf32x3", 2e-5)])
@pytest.mark.parametrize("case", range(len(PREP_CASES)))
def test_prep_chunk_images_leave_the_result_unchanged(gctx, gemm, tol, case):
    """The operand preparation with and without its k-chunks kept in shared memory (the two
    settings the autotuner chooses between, pinned with tk_plan_set_choice) writes the same slices,
    so the products agree bit for bit, and both match the oracle."""
    api = _api()
    la, lb = PREP_CASES[case]
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    xa, xb = wl.normal(31, oa.numel), wl.normal(32, ob.numel)
    cs, ref = ops.contract(oa, xa, (0,), (1,), ob, xb, (0,), (1,), (0,), (1,), tier="block")
    A, B = _tm(gctx, "U1", la), _tm(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, (0,), (1,), B, (0,), (1,), (0,), (1,), gemm=gemm)
    da, db = torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda()
    out = []
    for prep in (1, 2):
        api.set_choice(gctx, plan, prep=prep)
        out.append(_run(gctx, plan, da, db))
    assert torch.equal(out[0], out[1])
    assert rel_frobenius_per_block(cs, out[1].cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("gemm", ["ozaki", "tf32x3"])
def test_identity_product_shows_the_operand_split(gctx, gemm):
    """C = A I: with every B entry 0 or 1 (column scale 2, one digit 1/2, no TF32 remainder) the
    result is A's split representation itself, so the split's own error shows element by element.
    Ozaki BF16 (six digits): within (2^-43 + 2^-46) of the row's power-of-two scale, below
    2^-41 max|a_m.|.  3xTF32: hi + lo within 2^-23 |a| of a, plus one FP32 rounding of their sum in
    the accumulator, below 2^-21 |a|.  Entries spread over 2^+-20 inside each row, ragged tiles
    (M = 300, K = N = 100 in the wide sector; the 9-wide sector runs as double-float rows)."""
    api = _api()
    la = ([({0: 300, 1: 20}, False)], [({0: 100, 1: 9}, False)])
    lb = ([({0: 100, 1: 9}, False)], [({0: 100, 1: 9}, False)])
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    rng = np.random.default_rng(21)
    xa = wl.normal(9, oa.numel) * np.exp2(rng.integers(-20, 21, oa.numel).astype(float))
    xb = np.zeros(ob.numel)
    for _c, rows, cols, off in ob.blocks:
        assert rows == cols
        xb[off + np.arange(rows) * (rows + 1)] = 1.0
    cs, ref = ops.contract(oa, xa, (0,), (1,), ob, xb, (0,), (1,), (0,), (1,), tier="block")
    A, B = _tm(gctx, "U1", la), _tm(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, (0,), (1,), B, (0,), (1,), (0,), (1,), gemm=gemm)
    assert plan.tensor_flops > 0  # the wide sector is on the tensor-core path
    got = _run(gctx, plan, torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda()).cpu().numpy()
    for _c, rows, cols, off in cs.blocks:
        r = ref[off:off + rows * cols].reshape(cols, rows).T
        g = got[off:off + rows * cols].reshape(cols, rows).T
        if gemm == "ozaki":
            bound = 2.0 ** (-41) * np.abs(r).max(axis=1)[:, None]
        else:
            bound = 2.0 ** (-21) * np.abs(r)
        assert np.all(np.abs(g - r) <= bound)
        assert np.any(g != r)  # the split is not exact for these entries: the bound is what holds


@pytest.mark.parametrize("gemm,factor", [("ozaki", 8 * 2.0 ** (-42)), ("tf32x3", 2.0 ** (-17))])
@pytest.mark.parametrize("ea,eb", [(500, -500), (-600, -400), (600, 300)])
def test_scales_outside_the_fast_epilogue_range(gctx, ea, eb, gemm, factor):
    """Row scales near 2^ea and column scales near 2^eb, beyond the +-448 for which the epilogue
    skips its range checks: the checked path (and, for results near 2^-1000 or 2^1000, the exact
    slow conversion) must give the same accuracy as ordinary scales.  3xTF32 (11 + 11 bits per
    operand, FP32 accumulation) is held to a bound 2^25 times looser."""
    api = _api()
    la = ([({0: 130, 1: 20}, False)], [({0: 100, 1: 9}, False)])
    lb = ([({0: 100, 1: 9}, False)], [({0: 140, 1: 33}, False)])
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    rng = np.random.default_rng(11)
    xa = wl.normal(3, oa.numel) * np.exp2(ea + rng.integers(-8, 9, oa.numel).astype(float))
    xb = wl.normal(4, ob.numel) * np.exp2(eb + rng.integers(-8, 9, ob.numel).astype(float))
    cs, ref = ops.contract(oa, xa, (0,), (1,), ob, xb, (0,), (1,), (0,), (1,), tier="block")
    A, B = _tm(gctx, "U1", la), _tm(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, (0,), (1,), B, (0,), (1,), (0,), (1,), gemm=gemm)
    c = _run(gctx, plan, torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda())
    _elementwise_bound_check(oa, xa, ob, xb, cs, ref, c.cpu().numpy(), factor)


@pytest.mark.parametrize("slices", [2, 3, 4, 5])
def test_low_slice_counts(gctx, slices):
    """Fewer than four slices leave level accumulators unwritten (the epilogue's masked path); the
    error follows the digits kept: each operand entry within 2^(-7s) of its row's (column's)
    maximum, and the dropped slice pairs at most (s + 2) 2^(-7s) more per product, with scales up
    to twice the maxima (factor 4)."""
    api = _api()
    la = ([({0: 130, 1: 20}, False)], [({0: 100, 1: 9}, False)])
    lb = ([({0: 100, 1: 9}, False)], [({0: 140, 1: 33}, False)])
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    xa, xb = wl.normal(5, oa.numel), wl.normal(6, ob.numel)
    cs, ref = ops.contract(oa, xa, (0,), (1,), ob, xb, (0,), (1,), (0,), (1,), tier="block")
    A, B = _tm(gctx, "U1", la), _tm(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, (0,), (1,), B, (0,), (1,), (0,), (1,), gemm="ozaki", slices=slices)
    c = _run(gctx, plan, torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda())
    got = c.cpu().numpy()
    _elementwise_bound_check(oa, xa, ob, xb, cs, ref, got, 4 * (slices + 4) * 2.0 ** (-7 * slices))
    # and not far better than the digits allow: the error does shrink with the slice count
    assert rel_frobenius_per_block(cs, got, ref) > 2.0 ** (-7 * slices - 14)


TF32X3_TOL = 1e-5  # about FP32 accuracy: reported, not gated at the split-precision bar


def test_tf32x3_c0_and_heff(gctx):
    """3xTF32 (hi.hi + hi.lo + lo.hi on tcgen05 kind::tf32): about FP32 accuracy on C0 and on every
    step of the D = 1024 heff chain."""
    api = _api()
    v = {-2: 1, -1: 2, 0: 3, 1: 2, 2: 1}
    la = ([(v, False), (v, False)], [(v, False), (v, False)])
    lb = ([(v, False), (v, True)], [(v, False), (v, False)])
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    xa, xb = wl.normal(0, oa.numel), wl.normal(1, ob.numel)
    cs, ref = ops.contract(oa, xa, *wl.C0_SPEC[:2], ob, xb, *wl.C0_SPEC[2:], tier="dense")
    A, B = _tm(gctx, "U1", la), _tm(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, *wl.C0_SPEC[:2], B, *wl.C0_SPEC[2:], gemm="tf32x3")
    c = _run(gctx, plan, torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda())
    err = rel_frobenius_per_block(cs, c.cpu().numpy(), ref)
    assert 0 < err <= TF32X3_TOL
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(gctx, "U1", 1024, gemm="tf32x3")
    refs = oracle_heff("U1", 1024, tier="block")
    t = ch.steps[0].run(ch.dev["L"], ch.dev["x"])
    outs = [t]
    for i, other in ((1, "W"), (2, "W"), (3, "R")):
        t = ch.steps[i].run(t, ch.dev[other])
        outs.append(t)
    gctx.sync()
    for i, ((cs, rd), b) in enumerate(zip(refs, outs)):
        assert rel_frobenius_per_block(cs, b.cpu().numpy(), rd) <= TF32X3_TOL, i


def test_tf32x3_wide_range_and_split_k(gctx):
    """Rows and columns scaled by 2^(+-40) and K = 5000 (split across CTAs): per-row and
    per-column scales keep 3xTF32 at about FP32 accuracy relative to each row's and column's
    largest entries."""
    api = _api()
    la = ([({0: 130, 1: 20}, False)], [({0: 5000, 1: 9}, False)])
    lb = ([({0: 5000, 1: 9}, False)], [({0: 140, 1: 33}, False)])
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    rng = np.random.default_rng(10)
    xa = wl.normal(17, oa.numel) * np.exp2(rng.integers(-40, 41, oa.numel))
    xb = wl.normal(18, ob.numel) * np.exp2(rng.integers(-40, 41, ob.numel))
    cs, ref = ops.contract(oa, xa, (0,), (1,), ob, xb, (0,), (1,), (0,), (1,), tier="block")
    A, B = _tm(gctx, "U1", la), _tm(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, (0,), (1,), B, (0,), (1,), (0,), (1,), gemm="tf32x3")
    c = _run(gctx, plan, torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda())
    got = c.cpu().numpy()
    for (ca, ra, ka, oa_), (cb, rb, kb, ob_), (cc, rc, kc, oc) in zip(oa.blocks, ob.blocks, cs.blocks):
        am = xa[oa_:oa_ + ra * ka].reshape(ka, ra).T
        bm = xb[ob_:ob_ + rb * kb].reshape(kb, rb).T
        # hi and lo keep 22 bits: each operand entry is off by at most 2^-21 of its row's (column's)
        # scale 2^e <= 2 max; FP32 accumulation adds at most K 2^-24 of the running magnitude
        bound = (2 * 2 * 2.0 ** (-21) + 2.0 ** (-24) * 4) * ka * np.abs(am).max(axis=1)[:, None] * np.abs(bm).max(axis=0)[None, :]
        err = np.abs(got[oc:oc + rc * kc] - ref[oc:oc + rc * kc]).reshape(kc, rc).T
        assert np.all(err <= bound)


@pytest.mark.parametrize("gemm,tol", [("ozaki", SPLIT_TOL), ("tf32x3", 2e-5)])
def test_complex_split_precision(gctx, gemm, tol):
    """Complex tensors in the split-precision modes: four real products on the tensor cores,
    combined into the complex result; the complex heff chain against the oracle."""
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(gctx, "U1", 256, dtype="c128", gemm=gemm, seed=5)
    refs = oracle_heff("U1", 256, seed=5, tier="block", dtype="c128")
    t = ch.steps[0].run(ch.dev["L"], ch.dev["x"])
    outs = [t]
    for i, other in ((1, "W"), (2, "W"), (3, "R")):
        t = ch.steps[i].run(t, ch.dev[other])
        outs.append(t)
    gctx.sync()
    for i, ((cs, rd), b) in enumerate(zip(refs, outs)):
        assert ch.steps[i].out.blocks() == [(c, r, k, o) for c, r, k, o in cs.blocks]
        assert rel_frobenius_per_block(cs, b.cpu().numpy(), rd) <= tol, i


def test_complex_split_precision_su2_autotuned(gctx):
    """SU(2) complex L.x in Ozaki mode after autotuning (the real plan is tuned on the real parts)
    and replayed from a CUDA graph."""
    from paper_2508_10076_gb300.chain import LxContraction
    ch = LxContraction(gctx, "SU2", 256, dtype="c128", gemm="ozaki", seed=6)
    ch.autotune()
    graph, out, _ = ch.capture()
    graph.replay()
    torch.cuda.synchronize()
    cs, rd = oracle_heff("SU2", 256, seed=6, tier="block", dtype="c128", steps=1)[0]
    assert rel_frobenius_per_block(cs, out.cpu().numpy(), rd) <= SPLIT_TOL


def test_single_site_heff_split_precision(gctx):
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(gctx, "SU2", 256, sites=1, gemm="ozaki", seed=8)
    got = ch.run()
    gctx.sync()
    cs, rd = oracle_heff("SU2", 256, seed=8, tier="block", sites=1)[-1]
    assert rel_frobenius_per_block(cs, got.cpu().numpy(), rd) <= SPLIT_TOL


EDGE_CASES = [
    # (legs of A, legs of B): contraction of A's domain with B's codomain
    # an empty inner dimension (sector 1 has no K): zero block
    (([({0: 2, 1: 3}, False)], [({0: 3}, False)]), ([({0: 3}, False)], [({0: 2, 1: 1}, False)])),
    # single rows / columns and K = 1 (thin products on the double-float rows)
    (([({0: 1, 1: 1}, False)], [({0: 1, 1: 1}, False)]), ([({0: 1, 1: 1}, False)], [({0: 1, 1: 1}, False)])),
    # M just over one 128-row tile, N over a 128-column tile by 9, K crossing 32-deep chunks raggedly
    (([({0: 129, 1: 7}, False)], [({0: 33, 1: 70}, False)]), ([({0: 33, 1: 70}, False)], [({0: 137, 1: 16}, False)])),
]


@pytest.mark.parametrize("gemm", ["ozaki", "tf32x3"])
@pytest.mark.parametrize("case", range(len(EDGE_CASES)))
def test_split_precision_edge_cases(gctx, gemm, case):
    """Split-precision plans on degenerate and ragged shapes: every output entry written (no NaN
    left), values against the oracle within the mode's bound."""
    api = _api()
    la, lb = EDGE_CASES[case]
    A, B = _tm(gctx, "U1", la), _tm(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, (0,), (1,), B, (0,), (1,), (0,), (1,), gemm=gemm)
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    xa, xb = wl.normal(70 + case, oa.numel), wl.normal(80 + case, ob.numel)
    cs, ref = ops.contract(oa, xa, (0,), (1,), ob, xb, (0,), (1,), (0,), (1,), tier="block")
    got = _run(gctx, plan, torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda()).cpu().numpy()
    assert not np.isnan(got).any()
    assert rel_frobenius_per_block(cs, got, ref) <= (SPLIT_TOL if gemm == "ozaki" else 2e-5)


@pytest.mark.parametrize("planted", ["tiny", "huge", "mpo"])
def test_skinny_products_outside_the_double_float_window(gctx, planted):
    """The N <= 8 products of the split-precision modes run in double-float arithmetic, which keeps
    its precision only for A values in [2^-58, 2^96) and B values in [2^-20, 2^20).  Plant a few
    values outside those windows in one part of a long skinny product: the row blocks that meet
    them are redone in FP64 after the launch, the others keep their double-float results, and the
    whole output matches the oracle block by block."""
    api = _api()
    la = ([({0: 3000, 1: 2500}, False)], [({0: 4, 1: 4}, False)])   # A: M x K with K = 4
    lb = ([({0: 4, 1: 4}, False)], [({0: 4, 1: 3}, False)])         # B: K x N with N <= 4
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    xa, xb = wl.normal(21, oa.numel), wl.normal(22, ob.numel)
    if planted == "tiny":
        xa[100:104] = 2.0 ** -70 * np.array([1.0, -3.0, 0.5, 7.0])    # in the first row block only
    elif planted == "huge":
        xa[-5:] = 2.0 ** 100                                            # the last rows of the last sector
    else:
        xb[3] = 2.0 ** 30                                              # one MPO-side value
    cs, ref = ops.contract(oa, xa, (0,), (1,), ob, xb, (0,), (1,), (0,), (1,), tier="block")
    A, B = _tm(gctx, "U1", la), _tm(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, (0,), (1,), B, (0,), (1,), (0,), (1,), gemm="ozaki")
    c = _run(gctx, plan, torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda())
    got = c.cpu().numpy()
    assert np.isfinite(got).all()
    assert rel_frobenius_per_block(cs, got, ref) <= 1e-12
    # and row by row: every output row within the double-float bound of its own terms
    for (ca, ra, ka, oa_), (cb, rb, kb, ob_), (cc, rc, kc, oc) in zip(oa.blocks, ob.blocks, cs.blocks):
        am = xa[oa_:oa_ + ra * ka].reshape(ka, ra).T
        bm = xb[ob_:ob_ + rb * kb].reshape(kb, rb).T
        bound = 2.0 ** -40 * (np.abs(am) @ np.abs(bm))
        err = np.abs(got[oc:oc + rc * kc] - ref[oc:oc + rc * kc]).reshape(kc, rc).T
        assert np.all(err <= bound)
    c2 = _run(gctx, plan, torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda())
    assert torch.equal(c, c2)  # the flags are cleared for every call: same bits again
