"""CUDA path (libtk through the C ABI) against the CPU oracle, element by element.

Bars: integer/structure work bit-exact; abelian permutes are pure copies and must be bit-exact;
FP64 contractions within a relative Frobenius error of 1e-12 per block.
"""

import numpy as np
import pytest

from harness import oracle_heff, oracle_heff_inputs, ostruct, rel_frobenius_per_block
from oracle import ops
from paper_2508_10076_gb300 import build_library
from paper_2508_10076_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def gctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build_library()
    from paper_2508_10076_gb300 import api
    ctx = api.Context(0)
    yield ctx
    torch.cuda.synchronize()
    ctx.sync()


def _api():
    from paper_2508_10076_gb300 import api
    return api


def _lib_tmap(ctx, sym, legs):
    cod, dom = legs
    return ctx.tmap([ctx.space(sym, s, d) for s, d in cod], [ctx.space(sym, s, d) for s, d in dom])


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


PERMUTE_CASES = [
    # (sym, legs) -- several tiles, ragged tails, dual legs, every tile mode
    ("U1", ([({-2: 3, -1: 37, 0: 70, 1: 41, 2: 5}, False), ({-1: 1, 1: 1}, False)],
            [({-2: 3, -1: 37, 0: 70, 1: 41, 2: 5}, True), ({-1: 1, 1: 2}, True)])),
    ("U1", ([({-1: 3, 0: 2, 1: 4}, False), ({0: 33, 1: 17}, True), ({-1: 5, 2: 9}, False)],
            [({0: 40, 1: 7, 2: 3}, False)])),
    ("SU2", ([({0: 9, 1: 7, 2: 5, 3: 2}, False), ({1: 1}, False)], [({0: 6, 1: 8, 2: 4}, True), ({1: 1}, True)])),
    ("SU2", ([({1: 3, 2: 2}, True), ({0: 2, 2: 3}, False), ({1: 2}, False)], [({0: 5, 2: 2, 4: 1}, False)])),
    ("Z2", ([({0: 50, 1: 45}, False), ({0: 2, 1: 3}, True)], [({0: 31, 1: 29}, False), ({1: 4}, True)])),
    # Deligne products (labels a1 * 4096 + f(a2), layout in include/tk.h)
    ("U1xSU2", ([({4096 * -1 + 1: 9, 0: 20, 2: 7, 4096 + 1: 11}, False), ({4096 + 1: 1, -4096 + 1: 1}, False)],
                [({0: 12, 2: 5, 4096 + 1: 6, -4096 + 1: 6, 2 * 4096: 3}, True), ({4096 + 1: 1}, True)])),
    ("Z2xU1", ([({2047: 30, 2048 + 4096: 41, 2049: 17}, False), ({2049 + 4096: 2, 2047: 1}, True)],
               [({2048 + 4096: 25, 2048: 33, 2050 + 4096: 4}, False), ({2049: 2}, True)])),
]


def _perms(n, rng, k=6):
    out = []
    for _ in range(k):
        perm = list(rng.permutation(n))
        s = int(rng.integers(0, n + 1))
        out.append((tuple(perm[:s]), tuple(perm[s:])))
    return out


@pytest.mark.parametrize("case", range(len(PERMUTE_CASES)))
@pytest.mark.parametrize("dtype", ["f64", "c128"])
def test_permute_parity(gctx, case, dtype):
    api = _api()
    sym, legs = PERMUTE_CASES[case]
    ost = ostruct(sym, legs)
    lt = _lib_tmap(gctx, sym, legs)
    x = wl.normal_complex(case, ost.numel) if dtype == "c128" else wl.normal(case, ost.numel)
    xd = _dev(x)
    rng = np.random.default_rng(100 + case)
    perms = _perms(ost.nleg, rng)
    perms.append(((ost.nleg - 1,) + tuple(range(ost.nleg - 1))[:1], tuple(range(1, ost.nleg - 1))))
    for p, q in perms:
        if sorted(p + q) != list(range(ost.nleg)):
            continue
        os_, ref = ops.permute_block(ost, x, p, q)
        plan = api.permute_plan(gctx, lt, p, q, dtype=dtype)
        out = plan.output()
        assert out.blocks() == [(c, r, k, o) for c, r, k, o in os_.blocks]
        yd = torch.full((out.numel,), float("nan"), dtype=xd.dtype, device="cuda")
        api.permute(gctx, plan, xd, yd)
        gctx.sync()
        got = yd.cpu().numpy()
        if sym in ("SU2", "U1xSU2"):  # non-abelian: weighted sums of sources
            assert np.allclose(got, ref, rtol=1e-13, atol=1e-13), (p, q)
        else:
            assert np.array_equal(got, ref), (p, q)


VECTOR_TRANSPOSE_CASES = [
    # R-like environments (MPO leg of extent 2-4 leading on both sides, then two virtual legs
    # swapped): short-vector transpose tiles with ragged edges
    ("U1", ([({-2: 2, 0: 3, 2: 4}, False), ({-1: 37, 0: 50, 1: 41}, True)], [({-1: 19, 0: 50, 1: 33}, True)])),
    ("SU2", ([({0: 2, 2: 3}, False), ({1: 17, 3: 20, 5: 9}, True)], [({1: 17, 3: 20, 5: 9}, True)])),
]


@pytest.mark.parametrize("case", range(len(VECTOR_TRANSPOSE_CASES)))
@pytest.mark.parametrize("dtype", ["f64", "c128"])
def test_short_vector_transpose(gctx, case, dtype):
    """Permute (0, 2) <- (1,) of an R-like tensor: the short MPO leg moves as a vector while the
    virtual legs are transposed; every element against the oracle."""
    api = _api()
    sym, legs = VECTOR_TRANSPOSE_CASES[case]
    ost = ostruct(sym, legs)
    lt = _lib_tmap(gctx, sym, legs)
    x = wl.normal_complex(40 + case, ost.numel) if dtype == "c128" else wl.normal(40 + case, ost.numel)
    os_, ref = ops.permute_block(ost, x, (0, 2), (1,))
    plan = api.permute_plan(gctx, lt, (0, 2), (1,), dtype=dtype)
    st = plan.permute_stats(0)
    assert st["transpose_tasks"] > 0 and st["generic_elems"] < st["transpose_elems"]
    assert plan.output().blocks() == [(c, r, k, o) for c, r, k, o in os_.blocks]
    yd = torch.full((plan.output().numel,), float("nan"), dtype=torch.complex128 if dtype == "c128" else torch.float64,
                    device="cuda")
    api.permute(gctx, plan, _dev(x), yd)
    gctx.sync()
    got = yd.cpu().numpy()
    if sym == "SU2":
        assert np.allclose(got, ref, rtol=1e-13, atol=1e-13)
    else:
        assert np.array_equal(got, ref)


def test_c0_contraction_fp64(gctx):
    api = _api()
    v = {-2: 1, -1: 2, 0: 3, 1: 2, 2: 1}
    la = ([(v, False), (v, False)], [(v, False), (v, False)])
    lb = ([(v, False), (v, True)], [(v, False), (v, False)])
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    for seed in range(3):
        xa, xb = wl.normal(2 * seed, oa.numel), wl.normal(2 * seed + 1, ob.numel)
        cs, ref = ops.contract(oa, xa, *wl.C0_SPEC[:2], ob, xb, *wl.C0_SPEC[2:], tier="dense")
        A, B = _lib_tmap(gctx, "U1", la), _lib_tmap(gctx, "U1", lb)
        plan = api.contract_plan(gctx, A, *wl.C0_SPEC[:2], B, *wl.C0_SPEC[2:])
        assert plan.flops == 34362
        c = torch.full((plan.output().numel,), float("nan"), dtype=torch.float64, device="cuda")
        ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
        api.contract(gctx, plan, _dev(xa), _dev(xb), c, ws)
        gctx.sync()
        got = c.cpu().numpy()
        assert rel_frobenius_per_block(cs, got, ref) <= FP64_TOL


def test_su2_lx_contraction_fp64(gctx):
    """SU(2) L.x at sum n = 256 (full dimension 750): permutes with 6j recoupling + GEMMs."""
    from paper_2508_10076_gb300.chain import LxContraction
    lx = LxContraction(gctx, "SU2", 256)
    got = lx.run()
    gctx.sync()
    st, data = oracle_heff_inputs("SU2", 256)
    cs, ref = ops.contract(st["L"], data["L"], *wl.LX_SPEC[:2], st["x"], data["x"], *wl.LX_SPEC[2:],
                           tier="block")
    assert lx.step.out.blocks() == [(c, r, k, o) for c, r, k, o in cs.blocks]
    assert rel_frobenius_per_block(cs, got.cpu().numpy(), ref) <= FP64_TOL


def test_heff_chain_u1_d1024_fp64(gctx):
    """The two-site heff chain at D = 1024, every intermediate against the oracle block tier."""
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(gctx, "U1", 1024)
    ref = oracle_heff("U1", 1024, tier="block")
    t = ch.dev["x"]
    bufs = []
    t = ch.steps[0].run(ch.dev["L"], t)
    bufs.append(t)
    t = ch.steps[1].run(t, ch.dev["W"])
    bufs.append(t)
    t = ch.steps[2].run(t, ch.dev["W"])
    bufs.append(t)
    t = ch.steps[3].run(t, ch.dev["R"])
    bufs.append(t)
    gctx.sync()
    for i, ((cs, rd), b) in enumerate(zip(ref, bufs)):
        assert ch.steps[i].out.blocks() == [(c, r, k, o) for c, r, k, o in cs.blocks]
        assert rel_frobenius_per_block(cs, b.cpu().numpy(), rd) <= FP64_TOL, i


def test_heff_chain_complex(gctx):
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(gctx, "U1", 96, dtype="c128", seed=3)
    got = ch.run()
    gctx.sync()
    cs, rd = oracle_heff("U1", 96, seed=3, tier="block", dtype="c128")[-1]
    assert rel_frobenius_per_block(cs, got.cpu().numpy(), rd) <= FP64_TOL


def test_zero_blocks_when_inner_dimension_empty(gctx):
    api = _api()
    la = ([({0: 2, 1: 3}, False)], [({0: 3}, False)])
    lb = ([({0: 3}, False)], [({0: 2, 1: 1}, False)])
    A, B = _lib_tmap(gctx, "U1", la), _lib_tmap(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, (0,), (1,), B, (0,), (1,), (0,), (1,))
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    xa, xb = wl.normal(1, oa.numel), wl.normal(2, ob.numel)
    cs, ref = ops.contract(oa, xa, (0,), (1,), ob, xb, (0,), (1,), (0,), (1,), tier="block")
    c = torch.full((plan.output().numel,), float("nan"), dtype=torch.float64, device="cuda")
    api.contract(gctx, plan, _dev(xa), _dev(xb), c, None)
    gctx.sync()
    got = c.cpu().numpy()
    assert not np.isnan(got).any()
    assert rel_frobenius_per_block(cs, got, ref) <= FP64_TOL


def test_rank_one_and_trivial_extents(gctx):
    api = _api()
    legs = ([({0: 1}, False)], [])
    lt = _lib_tmap(gctx, "SU2", legs)
    plan = api.permute_plan(gctx, lt, (), (0,))
    x = torch.tensor([2.5], dtype=torch.float64, device="cuda")
    y = torch.empty(1, dtype=torch.float64, device="cuda")
    api.permute(gctx, plan, x, y)
    gctx.sync()
    ost = ostruct("SU2", legs)
    _, ref = ops.permute_block(ost, np.array([2.5]), (), (0,))
    assert np.allclose(y.cpu().numpy(), ref)


def test_workspace_too_small_is_an_error(gctx):
    api = _api()
    from paper_2508_10076_gb300.chain import LxContraction
    lx = LxContraction(gctx, "SU2", 32)
    c = lx.step.c
    small = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(api.TKError) as e:
        api.contract(gctx, lx.step.plan, lx.dev["L"], lx.dev["x"], c, small)
    assert e.value.code == 9


def test_runs_are_bitwise_deterministic(gctx):
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(gctx, "U1", 256)
    a = ch.run().clone()
    b = ch.run().clone()
    gctx.sync()
    assert torch.equal(a, b)
    assert gctx.launches > 0


@pytest.mark.parametrize("gemm", ["fp64", "ozaki"])
def test_cuda_graph_replay_matches_eager(gctx, gemm):
    """One heff application recorded as a CUDA graph replays to the same bits as eager launches."""
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(gctx, "U1", 512, gemm=gemm, seed=2)
    eager = ch.run().clone()
    graph, out, launches = ch.capture()
    assert launches > 0
    ch.dev["x"].mul_(1.0)  # same inputs
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)


def test_split_k_few_tiles_long_inner_dimension(gctx):
    """A handful of output tiles over K = 2000: the inner dimension is cut into parts summed in a
    fixed order by the last CTA to finish; the result matches the oracle and repeats bit for bit."""
    api = _api()
    la = ([({0: 64, 1: 40}, False)], [({0: 2000, 1: 700}, False)])
    lb = ([({0: 2000, 1: 700}, False)], [({0: 50, 1: 33}, False)])
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    xa, xb = wl.normal(11, oa.numel), wl.normal(12, ob.numel)
    cs, ref = ops.contract(oa, xa, (0,), (1,), ob, xb, (0,), (1,), (0,), (1,), tier="block")
    A, B = _lib_tmap(gctx, "U1", la), _lib_tmap(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, (0,), (1,), B, (0,), (1,), (0,), (1,))
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    outs = []
    for _ in range(3):
        c = torch.full((plan.output().numel,), float("nan"), dtype=torch.float64, device="cuda")
        api.contract(gctx, plan, _dev(xa), _dev(xb), c, ws)
        outs.append(c)
    gctx.sync()
    assert rel_frobenius_per_block(cs, outs[0].cpu().numpy(), ref) <= FP64_TOL
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


@pytest.mark.parametrize("sym,D", [("U1", 1024), ("SU2", 256)])
def test_single_site_heff_chain_fp64(gctx, sym, D):
    """Algorithm 11 (x' = L.x.W.R, three contractions): every intermediate against the oracle."""
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(gctx, sym, D, sites=1, seed=7)
    ref = oracle_heff(sym, D, seed=7, tier="block", sites=1)
    t = ch.steps[0].run(ch.dev["L"], ch.dev["x"])
    outs = [t.clone()]
    for i in (1, 2):
        t = ch.steps[i].run(t, ch.dev[ch.others[i]])
        outs.append(t.clone())
    gctx.sync()
    assert len(ch.steps) == 3
    for i, ((cs, rd), b) in enumerate(zip(ref, outs)):
        assert ch.steps[i].out.blocks() == [(c, r, k, o) for c, r, k, o in cs.blocks]
        assert rel_frobenius_per_block(cs, b.cpu().numpy(), rd) <= FP64_TOL, i


@pytest.mark.parametrize("dtype", ["f64", "c128"])
def test_adjoint_parity(gctx, dtype):
    """t^dagger on the GPU (block transposes on the permute kernels, conjugated for complex)
    against the oracle's dense definition, bit for bit (pure data movement)."""
    api = _api()
    for case, (sym, legs) in enumerate(PERMUTE_CASES):
        ost = ostruct(sym, legs)
        x = wl.normal_complex(30 + case, ost.numel) if dtype == "c128" else wl.normal(30 + case, ost.numel)
        os2, ref = ops.adjoint(ost, x, tier="dense")
        lt = _lib_tmap(gctx, sym, legs)
        plan = api.adjoint_plan(gctx, lt, dtype=dtype)
        assert plan.output().blocks() == [(c, r, k, o) for c, r, k, o in os2.blocks]
        xd = _dev(x)
        y = torch.full((plan.output().numel,), float("nan"), dtype=xd.dtype, device="cuda")
        api.permute(gctx, plan, xd, y)
        gctx.sync()
        _, blk = ops.adjoint(ost, x, tier="block")
        assert np.array_equal(y.cpu().numpy(), blk)
        assert np.allclose(y.cpu().numpy(), ref, atol=1e-12)


@pytest.mark.parametrize("gemm,tol", [("fp64", FP64_TOL), ("ozaki", 1e-10), ("tf32x3", 1e-10)])
def test_long_skinny_products(gctx, gemm, tol):
    """MPO-like products with N <= 8 over about a million rows (the shape of the heff chain's
    T.W steps at D = 4096): row blocks with several rows per thread, ragged last blocks, and inner
    dimensions 4 (full groups) and 7 (a group plus a tail).  The skinny products run in FP64 or in
    double-float in every mode, so all modes meet the FP64-class bound."""
    api = _api()
    la = ([({0: 1_000_003, 1: 950_001}, False)], [({0: 4, 1: 7}, False)])
    lb = ([({0: 4, 1: 7}, False)], [({0: 2, 1: 3}, False)])
    oa, ob = ostruct("U1", la), ostruct("U1", lb)
    xa, xb = wl.normal(21, oa.numel), wl.normal(22, ob.numel)
    cs, ref = ops.contract(oa, xa, (0,), (1,), ob, xb, (0,), (1,), (0,), (1,), tier="block")
    A, B = _lib_tmap(gctx, "U1", la), _lib_tmap(gctx, "U1", lb)
    plan = api.contract_plan(gctx, A, (0,), (1,), B, (0,), (1,), (0,), (1,), gemm=gemm)
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    c = torch.full((plan.output().numel,), float("nan"), dtype=torch.float64, device="cuda")
    api.contract(gctx, plan, _dev(xa), _dev(xb), c, ws)
    gctx.sync()
    assert rel_frobenius_per_block(cs, c.cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("gemm,tol", [("fp64", FP64_TOL), ("ozaki", 1e-10)])
def test_product_symmetry_contraction(gctx, gemm, tol):
    """U(1) x SU(2) environment times two-site-like tensor (the L.x step with charge x spin
    sectors): block structure bit-exact and values within the FP64 / split-precision bounds."""
    from oracle.symmetry import U1xSU2
    api = _api()
    P = U1xSU2.pair
    vs = {P(q, t): n for (q, t), n in {(-2, 0): 20, (-1, 1): 31, (0, 0): 40, (0, 2): 23, (1, 1): 29,
                                         (2, 0): 17, (1, 3): 9, (-1, 3): 8}.items()}
    ps = {P(1, 1): 1, P(-1, 1): 1}
    ws = {P(0, 0): 2, P(0, 2): 1}
    la = ([(vs, False)], [(vs, False), (ws, False)])
    lx = ([(vs, False), (ps, False)], [(vs, False), (ps, True)])
    oa, ox = ostruct("U1xSU2", la), ostruct("U1xSU2", lx)
    xa, xx = wl.normal(31, oa.numel), wl.normal(32, ox.numel)
    spec = ((0, 2), (1,), (0,), (1, 2, 3), (0, 1, 2, 3, 4), ())
    cs, ref = ops.contract(oa, xa, *spec[:2], ox, xx, *spec[2:], tier="block")
    A, X = _lib_tmap(gctx, "U1xSU2", la), _lib_tmap(gctx, "U1xSU2", lx)
    plan = api.contract_plan(gctx, A, *spec[:2], X, *spec[2:], gemm=gemm)
    assert plan.output().blocks() == [(c, r, k, o) for c, r, k, o in cs.blocks]
    ws_ = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    c = torch.full((plan.output().numel,), float("nan"), dtype=torch.float64, device="cuda")
    api.contract(gctx, plan, _dev(xa), _dev(xx), c, ws_)
    gctx.sync()
    assert rel_frobenius_per_block(cs, c.cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("gemm,tol", [("fp64", FP64_TOL), ("ozaki", 1e-10)])
def test_heff_chain_product_symmetry(gctx, gemm, tol):
    """The two-site heff chain with U(1) x SU(2) (charge x spin) sectors, reduced virtual
    dimension 256: every intermediate against the oracle block tier."""
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(gctx, "U1xSU2", 256, gemm=gemm, seed=3)
    ref = oracle_heff("U1xSU2", 256, seed=3, tier="block")
    t = ch.steps[0].run(ch.dev["L"], ch.dev["x"])
    outs = [t]
    for i, other in ((1, "W"), (2, "W"), (3, "R")):
        t = ch.steps[i].run(t, ch.dev[other])
        outs.append(t)
    gctx.sync()
    for i, ((cs, rd), b) in enumerate(zip(ref, outs)):
        assert ch.steps[i].out.blocks() == [(c, r, k, o) for c, r, k, o in cs.blocks]
        assert rel_frobenius_per_block(cs, b.cpu().numpy(), rd) <= tol, i


@pytest.mark.parametrize("gemm,tol", [("fp64", FP64_TOL), ("ozaki", 1e-10)])
def test_heff_chain_su2_heisenberg(gctx, gemm, tol):
    """The SU(2) two-site heff chain with the Heisenberg MPO (stored reduced entries, pinned
    against the oracle's projection of the dense MPO): every intermediate against the oracle."""
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(gctx, "SU2", 256, gemm=gemm, seed=4, mpo="heisenberg")
    ref = oracle_heff("SU2", 256, seed=4, tier="block", mpo="heisenberg")
    t = ch.steps[0].run(ch.dev["L"], ch.dev["x"])
    outs = [t]
    for i, other in ((1, "W"), (2, "W"), (3, "R")):
        t = ch.steps[i].run(t, ch.dev[other])
        outs.append(t)
    gctx.sync()
    for i, ((cs, rd), b) in enumerate(zip(ref, outs)):
        assert ch.steps[i].out.blocks() == [(c, r, k, o) for c, r, k, o in cs.blocks]
        assert rel_frobenius_per_block(cs, b.cpu().numpy(), rd) <= tol, i


@pytest.mark.parametrize("gemm,tol", [("fp64", FP64_TOL), ("ozaki", 1e-10)])
def test_compose_parity(gctx, gemm, tol):
    """Composition A o B (Sec. 2.3): SU(2) blocks, against the oracle's block composition."""
    api = _api()
    v = {0: 40, 1: 70, 2: 55, 3: 20}
    p = {1: 1}
    la = ([(v, False), (p, False)], [(v, False)])
    lb = ([(v, False)], [(v, False), (p, True)])
    oa, ob = ostruct("SU2", la), ostruct("SU2", lb)
    xa, xb = wl.normal(91, oa.numel), wl.normal(92, ob.numel)
    cs, ref = ops.compose_block(oa, xa, ob, xb)
    A, B = _lib_tmap(gctx, "SU2", la), _lib_tmap(gctx, "SU2", lb)
    plan = api.compose_plan(gctx, A, B, gemm=gemm)
    assert plan.output().blocks() == [(c, r, k, o) for c, r, k, o in cs.blocks]
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    c = torch.full((plan.output().numel,), float("nan"), dtype=torch.float64, device="cuda")
    api.contract(gctx, plan, _dev(xa), _dev(xb), c, ws)
    gctx.sync()
    assert rel_frobenius_per_block(cs, c.cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("dtype", ["f64", "c128"])
@pytest.mark.parametrize("gemm,tol", [("fp64", FP64_TOL), ("ozaki", 1e-10)])
@pytest.mark.parametrize("sym", ["Z2", "Z2xU1"])
def test_z2_family_contraction(gctx, sym, gemm, tol, dtype):
    """Z2 and Z2 x U(1) (parity x charge, bosonic braiding) sectors through the L.x contraction:
    block structure bit-exact, values against the oracle block tier in FP64 and split precision,
    real and complex."""
    from oracle.symmetry import Z2xU1
    api = _api()
    if sym == "Z2":
        vs, ps, ws = {0: 70, 1: 55}, {0: 1, 1: 1}, {0: 3, 1: 2}
    else:
        P = Z2xU1.pair
        vs = {P(a, q): n for (a, q), n in {(0, -2): 11, (1, -1): 25, (0, 0): 38, (1, 0): 14, (0, 1): 27,
                                             (1, 1): 30, (0, 2): 9}.items()}
        ps = {P(1, 1): 1, P(1, -1): 1, P(0, 0): 1}
        ws = {P(0, 0): 2, P(0, 2): 1, P(0, -2): 1}
    la = ([(vs, False)], [(vs, False), (ws, False)])
    lx = ([(vs, False), (ps, False)], [(vs, False), (ps, True)])
    oa, ox = ostruct(sym, la), ostruct(sym, lx)
    gen = wl.normal_complex if dtype == "c128" else wl.normal
    xa, xx = gen(41, oa.numel), gen(42, ox.numel)
    spec = ((0, 2), (1,), (0,), (1, 2, 3), (0, 1, 2, 3, 4), ())
    cs, ref = ops.contract(oa, xa, *spec[:2], ox, xx, *spec[2:], tier="block")
    A, X = _lib_tmap(gctx, sym, la), _lib_tmap(gctx, sym, lx)
    plan = api.contract_plan(gctx, A, *spec[:2], X, *spec[2:], dtype=dtype, gemm=gemm)
    assert plan.output().blocks() == [(c, r, k, o) for c, r, k, o in cs.blocks]
    ws_ = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    tdt = torch.complex128 if dtype == "c128" else torch.float64
    c = torch.full((plan.output().numel,), float("nan"), dtype=tdt, device="cuda")
    api.contract(gctx, plan, _dev(xa), _dev(xx), c, ws_)
    gctx.sync()
    assert rel_frobenius_per_block(cs, c.cpu().numpy(), ref) <= tol


def test_heff_chain_host_to_host(gctx):
    """HeffChain.run_host (pinned host inputs, W and R copied beside the first contraction, x'
    read back) gives the device path's bits, eagerly and replayed from a CUDA graph."""
    from paper_2508_10076_gb300.chain import HeffChain, capture_graph
    ch = HeffChain(gctx, "U1", 128, seed=6)
    ref = ch.run().clone()
    gctx.sync()
    host = {k: ch.dev[k].cpu().pin_memory() for k in ("x", "L", "W", "R")}
    for k in host:  # the call must copy every input itself
        ch.dev[k].zero_()
    out = torch.empty(ref.numel(), dtype=ref.dtype).pin_memory()
    ch.run_host(host, out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref.cpu())
    graph, _, _ = capture_graph(gctx, lambda: ch.run_host(host, out))
    out.zero_()
    for k in host:
        ch.dev[k].zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref.cpu())
