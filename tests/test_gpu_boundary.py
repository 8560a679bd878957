"""The context's device-memory boundary on the GPU: every library allocation goes through the
caller's hooks (counted here), a budget refuses plans whose tables do not fit (TK_ERR_BUDGET),
typed tensor-map upload / download round-trip the blocks, and a NULL stream runs on the context's
stream.  Results are checked against the oracle."""

import ctypes as C
import gc

import numpy as np
import pytest

from harness import ostruct, rel_frobenius_per_block
from oracle import ops
from paper_2508_10076_gb300 import build_library
from paper_2508_10076_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TK_ERR_BUDGET = 11


class CountingTorchAllocator:
    """Allocator hooks over PyTorch's caching allocator that count live blocks and bytes."""

    def __init__(self):
        self.live = {}
        self.calls = 0

    def alloc(self, nbytes):
        p = int(torch.cuda.caching_allocator_alloc(nbytes, 0, torch.cuda.current_stream()))
        self.live[p] = nbytes
        self.calls += 1
        return p

    def free(self, ptr, nbytes):
        assert self.live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)


def _lx(ctx, sym, D):
    V, P, W = wl.heff_spaces(sym, D)
    legs = wl.heff_legs(V, P, W)
    tm = {k: ctx.tmap([ctx.space(sym, s, d) for s, d in legs[k][0]], [ctx.space(sym, s, d) for s, d in legs[k][1]])
          for k in ("L", "x")}
    return legs, tm


@pytest.mark.parametrize("sym,D,dtype,gemm", [("U1", 256, "f64", "fp64"), ("SU2", 64, "f64", "ozaki"),
                                              ("U1", 128, "c128", "ozaki")])
def test_every_library_allocation_goes_through_the_hooks(sym, D, dtype, gemm):
    assert torch.cuda.is_available()
    build_library()
    from paper_2508_10076_gb300 import api
    hooks = CountingTorchAllocator()
    ctx = api.Context(0, allocator=(hooks.alloc, hooks.free))
    assert hooks.calls == 1 and ctx.memory()["allocations"] == 1  # the status word
    legs, tm = _lx(ctx, sym, D)
    plan = api.contract_plan(ctx, tm["L"], *wl.LX_SPEC[:2], tm["x"], *wl.LX_SPEC[2:], dtype=dtype, gemm=gemm)
    mem = ctx.memory()
    assert mem["allocations"] == len(hooks.live) > 1
    assert mem["library_bytes"] == sum(hooks.live.values())
    rnd = wl.normal_complex if dtype == "c128" else wl.normal
    a, b = rnd(5, tm["L"].numel), rnd(6, tm["x"].numel)
    tdt = torch.complex128 if dtype == "c128" else torch.float64
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    out = plan.output()
    c = torch.full((out.numel,), float("nan"), dtype=tdt, device="cuda")
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    api.contract(ctx, plan, ad, bd, c, ws)
    ctx.sync()
    cs, ref = ops.contract(ostruct(sym, legs["L"]), a, *wl.LX_SPEC[:2], ostruct(sym, legs["x"]), b,
                           *wl.LX_SPEC[2:], tier="block")
    assert rel_frobenius_per_block(cs, c.cpu().numpy(), ref) <= (1e-12 if gemm == "fp64" else 1e-10)
    # autotuning rebuilds the tables through the hooks too
    api.autotune(ctx, plan, ad, bd, c, ws)
    assert ctx.memory()["library_bytes"] == sum(hooks.live.values())
    del plan, out, tm
    ctx.close()
    gc.collect()
    assert hooks.live == {}, "every allocation is given back through the free hook"


def test_budget_refuses_plan_tables_that_do_not_fit():
    build_library()
    from paper_2508_10076_gb300 import api
    ctx = api.Context(0)
    ctx.set_budget(ctx.memory()["library_bytes"] + 64)
    _, tm = _lx(ctx, "U1", 256)
    with pytest.raises(api.TKError) as e:
        api.contract_plan(ctx, tm["L"], *wl.LX_SPEC[:2], tm["x"], *wl.LX_SPEC[2:])
    assert e.value.code == TK_ERR_BUDGET
    ctx.set_budget(0)
    plan = api.contract_plan(ctx, tm["L"], *wl.LX_SPEC[:2], tm["x"], *wl.LX_SPEC[2:])
    used = ctx.memory()["library_bytes"]
    ctx.set_budget(used + 1000)
    ctx.reserve(1000)
    with pytest.raises(api.TKError) as e:
        ctx.alloc(256)
    assert e.value.code == TK_ERR_BUDGET
    ctx.release(1000)
    p = ctx.alloc(256)
    assert ctx.memory()["library_bytes"] == used + 256
    ctx.free(p)
    assert plan.workspace_bytes > 0


def test_tmap_upload_download_round_trip_and_context_stream():
    build_library()
    from paper_2508_10076_gb300 import api
    from paper_2508_10076_gb300._abi import load
    s = torch.cuda.Stream()
    ctx = api.Context(0, stream=s)
    legs, tm = _lx(ctx, "SU2", 48)
    host = wl.normal_complex(9, tm["x"].numel)
    dev = ctx.alloc(host.nbytes)
    tm["x"].upload(host, dev, dtype="c128", stream=s)
    back = np.zeros_like(host)
    tm["x"].download(dev, back, dtype="c128", stream=s)
    s.synchronize()
    assert np.array_equal(back, host)
    ctx.free(dev)
    # a contraction launched with a NULL stream runs on the context's stream
    plan = api.contract_plan(ctx, tm["L"], *wl.LX_SPEC[:2], tm["x"], *wl.LX_SPEC[2:])
    a, b = wl.normal(1, tm["L"].numel), wl.normal(2, tm["x"].numel)
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    c = torch.full((plan.output().numel,), float("nan"), dtype=torch.float64, device="cuda")
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    rc = load().tk_contract(ctx._h, plan._h, C.c_void_p(ad.data_ptr()), C.c_void_p(bd.data_ptr()),
                            C.c_void_p(c.data_ptr()), C.c_void_p(ws.data_ptr()), C.c_size_t(ws.numel()), None)
    assert rc == 0
    ctx.sync(s)
    cs, ref = ops.contract(ostruct("SU2", legs["L"]), a, *wl.LX_SPEC[:2], ostruct("SU2", legs["x"]), b,
                           *wl.LX_SPEC[2:], tier="block")
    assert rel_frobenius_per_block(cs, c.cpu().numpy(), ref) <= 1e-12


def test_fp64_peak_probe_is_plausible():
    """The FP64 roofline denominator: a register-only FMA loop on every SM for the requested time.
    GB300's FP64 pipe retires 2 FMA per clock per SM (152 SMs, up to 2.07 GHz): 1.26 TFLOP/s."""
    build_library()
    from paper_2508_10076_gb300 import api
    ctx = api.Context(0)
    tflops, ms = api.probe_fp64_peak(ctx, seconds=0.2)
    assert 0.6 < tflops < 1.3
    assert 150 < ms < 260
