"""tk_contract_batch: many requests whose stages share launches give, for every request, the
bits tk_contract gives for that request alone (same tiles, same order of operations), and each
request's result matches the oracle's block-tier contraction (Algorithm 8) at the tolerance of
its GEMM mode."""

import numpy as np
import pytest

from harness import ostruct, rel_frobenius_per_block
from oracle import ops
from paper_2508_10076_gb300 import build_library
from paper_2508_10076_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ozaki": 1e-10, "tf32x3": 2e-5}


@pytest.fixture(scope="module")
def gctx():
    assert torch.cuda.is_available()
    build_library()
    from paper_2508_10076_gb300 import api
    ctx = api.Context(0)
    yield ctx
    ctx.sync()


def _tm(ctx, sym, legs):
    cod, dom = legs
    return ctx.tmap([ctx.space(sym, s, d) for s, d in cod], [ctx.space(sym, s, d) for s, d in dom])


def _requests(ctx, dtype, seed0, gemm="fp64", with_oracle=False):
    """(plan, A data, B data) for a mix of shapes: U(1) and SU(2) L.x, C0, a zero-block case,
    and one shape twice (two requests sharing a plan).  with_oracle also returns, per request,
    the oracle's arguments (structures, host data and the contraction's index lists)."""
    from paper_2508_10076_gb300 import api
    reqs, oargs = [], []
    rnd = wl.normal_complex if dtype == "c128" else wl.normal
    tdt = torch.complex128 if dtype == "c128" else torch.float64
    for k, (sym, D) in enumerate([("U1", 256), ("SU2", 96), ("U1", 256), ("U1", 96), ("SU2", 32)]):
        V, P, W = wl.heff_spaces(sym, D)
        legs = wl.heff_legs(V, P, W)
        L, x = _tm(ctx, sym, legs["L"]), _tm(ctx, sym, legs["x"])
        plan = api.contract_plan(ctx, L, *wl.LX_SPEC[:2], x, *wl.LX_SPEC[2:], dtype=dtype, gemm=gemm)
        reqs.append((plan, rnd(seed0 + 2 * k, L.numel), rnd(seed0 + 2 * k + 1, x.numel)))
        oargs.append((ostruct(sym, legs["L"]), ostruct(sym, legs["x"]), wl.LX_SPEC))
    v = {-2: 1, -1: 2, 0: 3, 1: 2, 2: 1}
    legs_a = ([(v, False), (v, False)], [(v, False), (v, False)])
    legs_b = ([(v, False), (v, True)], [(v, False), (v, False)])
    A, B = _tm(ctx, "U1", legs_a), _tm(ctx, "U1", legs_b)
    plan = api.contract_plan(ctx, A, *wl.C0_SPEC[:2], B, *wl.C0_SPEC[2:], dtype=dtype, gemm=gemm)
    reqs.append((plan, rnd(seed0 + 20, A.numel), rnd(seed0 + 21, B.numel)))
    oargs.append((ostruct("U1", legs_a), ostruct("U1", legs_b), wl.C0_SPEC))
    legs_a = ([({0: 2, 1: 3}, False)], [({0: 3}, False)])
    legs_b = ([({0: 3}, False)], [({0: 2, 1: 1}, False)])
    A, B = _tm(ctx, "U1", legs_a), _tm(ctx, "U1", legs_b)
    spec = ((0,), (1,), (0,), (1,), (0,), (1,))
    plan = api.contract_plan(ctx, A, *spec[:2], B, *spec[2:], dtype=dtype, gemm=gemm)
    reqs.append((plan, rnd(seed0 + 22, A.numel), rnd(seed0 + 23, B.numel)))
    oargs.append((ostruct("U1", legs_a), ostruct("U1", legs_b), spec))
    dev = [(p, torch.from_numpy(np.ascontiguousarray(a)).to("cuda", tdt),
            torch.from_numpy(np.ascontiguousarray(b)).to("cuda", tdt)) for p, a, b in reqs]
    if with_oracle:
        return dev, tdt, [(oa, a, ob, b, spec) for (oa, ob, spec), (_, a, b) in zip(oargs, reqs)]
    return dev, tdt


@pytest.mark.parametrize("dtype,gemm", [("f64", "fp64"), ("c128", "fp64"), ("f64", "ozaki"), ("f64", "tf32x3")])
def test_batch_equals_each_request_alone(gctx, dtype, gemm):
    """Split-precision batches pack every request's double-float rows into one launch and its
    tensor-core products into one launch per (tile width, slice count): still the bits of each
    request alone, and each request within its mode's tolerance of the oracle."""
    from paper_2508_10076_gb300 import api
    reqs, tdt, oracle_args = _requests(gctx, dtype, 40, gemm, with_oracle=True)
    alone, outs, wss = [], [], []
    for plan, a, b in reqs:
        c = torch.full((plan.output().numel,), float("nan"), dtype=tdt, device="cuda")
        ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
        api.contract(gctx, plan, a, b, c, ws)
        alone.append(c)
        outs.append(torch.full_like(c, float("nan")))
        wss.append(torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda"))
    api.contract_batch(gctx, [r[0] for r in reqs], [r[1] for r in reqs], [r[2] for r in reqs], outs, wss)
    gctx.sync()
    for i, (x, y) in enumerate(zip(alone, outs)):
        assert torch.equal(x, y), i
    for i, ((oa, a, ob, b, spec), y) in enumerate(zip(oracle_args, outs)):
        cs, ref = ops.contract(oa, a, *spec[:2], ob, b, *spec[2:], tier="block")
        assert rel_frobenius_per_block(cs, y.cpu().numpy(), ref) <= TOL[gemm], i


def test_batch_rejects_mixed_modes_and_small_workspace(gctx):
    from paper_2508_10076_gb300 import api
    reqs, tdt = _requests(gctx, "f64", 60)
    plan, a, b = reqs[0]
    c = torch.empty(plan.output().numel, dtype=tdt, device="cuda")
    small = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(api.TKError) as e:
        api.contract_batch(gctx, [plan], [a], [b], [c], [small])
    assert e.value.code == 9
    V, P, W = wl.heff_spaces("U1", 256)
    legs = wl.heff_legs(V, P, W)
    L, x = _tm(gctx, "U1", legs["L"]), _tm(gctx, "U1", legs["x"])
    oz = api.contract_plan(gctx, L, *wl.LX_SPEC[:2], x, *wl.LX_SPEC[2:], gemm="ozaki")
    ws = torch.empty(max(1, oz.workspace_bytes), dtype=torch.uint8, device="cuda")
    ws64 = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    with pytest.raises(api.TKError) as e:  # mixed gemm modes
        api.contract_batch(gctx, [plan, oz], [a, a], [b, b], [c, c], [ws64, ws])
    assert e.value.code == 7
    cz = api.contract_plan(gctx, L, *wl.LX_SPEC[:2], x, *wl.LX_SPEC[2:], dtype="c128", gemm="ozaki")
    wsz = torch.empty(max(1, cz.workspace_bytes), dtype=torch.uint8, device="cuda")
    cc = torch.empty(cz.output().numel, dtype=torch.complex128, device="cuda")
    az = torch.zeros(L.numel, dtype=torch.complex128, device="cuda")
    bz = torch.zeros(x.numel, dtype=torch.complex128, device="cuda")
    with pytest.raises(api.TKError) as e:  # complex split precision runs one by one
        api.contract_batch(gctx, [cz], [az], [bz], [cc], [wsz])
    assert e.value.code == 7
    api.contract_batch(gctx, [], [], [], [], [])  # empty batch: no-op
