"""tk_contract_noalloc: the contraction for callers that cannot allocate device memory.

Such callers (programs whose device memory belongs to another framework's allocator, serving
loops that must not take the synchronisation a cudaMalloc can cause, plug-ins that are handed
only their buffers) get the permuted operands and intermediates in a scratch array built into
libtk.  These tests call it through the C ABI and compare it with tk_contract, which takes a
caller-allocated workspace, and with the oracle.  The array is shared by every call and keeps
the previous call's contents, so the calls run back to back with different plans in between:
FP64, split precision (Ozaki BF16 and 3xTF32, whose scale arrays, slices and split-K counters live
in the scratch) and complex data, each on two calls in a row.  An oversized plan is refused.
"""

import numpy as np
import pytest

from harness import oracle_heff, ostruct, rel_frobenius_per_block
from oracle import ops
from paper_2508_10076_gb300 import build_library
from paper_2508_10076_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ozaki": 1e-10, "tf32x3": 2e-5}  # the parity tests' per-block tolerances


@pytest.fixture(scope="module")
def nctx():
    assert torch.cuda.is_available(), "needs a CUDA device"
    build_library()
    from paper_2508_10076_gb300 import api
    return api.Context(0)


def _tm(ctx, sym, legs):
    cod, dom = legs
    return ctx.tmap([ctx.space(sym, s, d) for s, d in cod], [ctx.space(sym, s, d) for s, d in dom])


def _run_both(ctx, plan, a, b, tdt):
    """(tk_contract with its own workspace, tk_contract_noalloc) on the same inputs, outputs
    NaN-poisoned beforehand."""
    from paper_2508_10076_gb300 import api
    n = plan.output().numel
    ref = torch.full((n,), float("nan"), dtype=tdt, device="cuda")
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    api.contract(ctx, plan, a, b, ref, ws)
    got = torch.full((n,), float("nan"), dtype=tdt, device="cuda")
    api.contract_noalloc(ctx, plan, a, b, got)
    ctx.sync()
    return ref, got


def _lx_case(ctx, sym, D, dtype, gemm, seed):
    """(plan, device inputs, oracle's result) of one seeded L.x contraction."""
    from paper_2508_10076_gb300 import api
    V, P, W = wl.heff_spaces(sym, D)
    legs = wl.heff_legs(V, P, W)
    L, x = _tm(ctx, sym, legs["L"]), _tm(ctx, sym, legs["x"])
    plan = api.contract_plan(ctx, L, *wl.LX_SPEC[:2], x, *wl.LX_SPEC[2:], dtype=dtype, gemm=gemm)
    rnd = wl.normal_complex if dtype == "c128" else wl.normal
    a, b = rnd(seed, L.numel), rnd(seed + 1, x.numel)
    cs, ref = ops.contract(ostruct(sym, legs["L"]), a, *wl.LX_SPEC[:2], ostruct(sym, legs["x"]), b,
                           *wl.LX_SPEC[2:], tier="block")
    tdt = torch.complex128 if dtype == "c128" else torch.float64
    return plan, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), cs, ref, tdt


# Run in this order on one context: every case follows a different plan's call, and the split-
# precision and complex cases find the array holding another plan's data.
CASES = [("SU2", 96, "f64", "fp64"), ("U1", 256, "f64", "ozaki"), ("U1", 256, "c128", "fp64"),
         ("U1", 256, "c128", "ozaki"), ("SU2", 64, "f64", "tf32x3"), ("U1", 256, "f64", "fp64")]


def test_noalloc_matches_workspace_contract_and_oracle_across_plans(nctx):
    from paper_2508_10076_gb300 import api
    limit = api.noalloc_scratch_bytes()
    for k, (sym, D, dtype, gemm) in enumerate(CASES):
        for call in range(2):  # two calls in a row, different data
            plan, a, b, cs, ref, tdt = _lx_case(nctx, sym, D, dtype, gemm, seed=100 * k + 10 * call)
            assert 0 < plan.workspace_bytes <= limit
            want, got = _run_both(nctx, plan, a, b, tdt)
            g = got.cpu().numpy()
            assert not np.isnan(g).any(), (sym, D, dtype, gemm, call)
            assert torch.equal(got, want), (sym, D, dtype, gemm, call)
            assert rel_frobenius_per_block(cs, g, ref) <= TOL[gemm], (sym, D, dtype, gemm, call)


def test_noalloc_heff_step_with_every_operand_permuted(nctx):
    """T2 = T1 W of the U(1) two-site chain: both operands and the result are permuted (three
    scratch regions in use); the oracle's T1 is the input of both sides."""
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(nctx, "U1", 256)
    step = ch.steps[1]
    (t1s, t1d), (t2s, t2d) = oracle_heff("U1", 256, seed=0, tier="block", steps=2)
    t1 = torch.from_numpy(np.ascontiguousarray(t1d)).cuda()
    for scale in (1.0, -0.5):
        want, got = _run_both(nctx, step.plan, t1 * scale, ch.dev["W"], torch.float64)
        assert torch.equal(got, want)
        assert rel_frobenius_per_block(t2s, got.cpu().numpy(), scale * t2d) <= TOL["fp64"]


def test_noalloc_refuses_plans_larger_than_its_scratch(nctx):
    from paper_2508_10076_gb300 import api
    V = {q: 100 for q in (-1, 0, 1)}
    s = nctx.space("U1", V)
    A = nctx.tmap([s, s], [s])
    B = nctx.tmap([s], [s, s])
    plan = api.contract_plan(nctx, A, (0,), (1, 2), B, (1, 0), (2,), (0,), (1,))
    assert plan.workspace_bytes > api.noalloc_scratch_bytes()
    # real, correctly sized buffers: the refusal must come before any launch, but nothing here
    # relies on that for memory safety
    a = torch.zeros(A.numel, dtype=torch.float64, device="cuda")
    b = torch.zeros(B.numel, dtype=torch.float64, device="cuda")
    c = torch.zeros(plan.output().numel, dtype=torch.float64, device="cuda")
    launches = nctx.launches
    with pytest.raises(api.TKError) as e:
        api.contract_noalloc(nctx, plan, a, b, c)
    assert e.value.code == 9
    assert nctx.launches == launches
