"""tk_contract_noalloc: the contraction for callers that cannot allocate device memory.

Such callers (programs whose device memory belongs to another framework's allocator, serving
loops that must not take the synchronisation a cudaMalloc can cause, plug-ins that are handed
only their buffers) get the permuted operands and intermediates in a scratch array built into
libtk.  These tests call it through the C ABI and compare it with tk_contract, which takes a
caller-allocated workspace, on two calls in a row with different data (the array keeps the
previous call's contents), and check that an oversized plan is refused.
"""

import numpy as np
import pytest

from harness import rel_frobenius_per_block
from paper_2508_10076_gb300 import build_library
from paper_2508_10076_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 per-block tolerance of the parity tests


@pytest.fixture(scope="module")
def nctx():
    assert torch.cuda.is_available(), "needs a CUDA device"
    build_library()
    from paper_2508_10076_gb300 import api
    return api.Context(0)


def _blocks(tm):
    return tm.blocks()


class _Struct:
    def __init__(self, blocks):
        self.blocks = blocks


def _compare(ctx, plan, a, b, c_ref_like):
    from paper_2508_10076_gb300 import api
    ref = torch.full_like(c_ref_like, float("nan"))
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    api.contract(ctx, plan, a, b, ref, ws)
    got = torch.full_like(c_ref_like, float("nan"))
    api.contract_noalloc(ctx, plan, a, b, got)
    ctx.sync()
    st = _Struct(plan.output().blocks())
    g, r = got.cpu().numpy(), ref.cpu().numpy()
    assert not np.isnan(g).any()
    return rel_frobenius_per_block(st, g, r)


@pytest.mark.parametrize("sym,D", [("U1", 256), ("SU2", 96)])
def test_noalloc_matches_workspace_contract_twice(nctx, sym, D):
    from paper_2508_10076_gb300 import api
    from paper_2508_10076_gb300.chain import HeffChain, LxContraction
    if sym == "U1":
        ch = HeffChain(nctx, sym, D)
        step = ch.steps[1]                      # T2 = T1 W: both operands permuted, output too
        t1 = ch.steps[0].run(ch.dev["L"], ch.dev["x"]).clone()
        inputs = [(t1, ch.dev["W"]), (t1 * -0.5 + 1.0, ch.dev["W"])]
    else:
        lx = LxContraction(nctx, sym, D)
        step = lx.step
        x2 = torch.from_numpy(wl.normal(77, lx.tm["x"].numel)).cuda()
        inputs = [(lx.dev["L"], lx.dev["x"]), (lx.dev["L"], x2)]
    assert 0 < step.plan.workspace_bytes <= api.NOALLOC_SCRATCH_BYTES
    for a, b in inputs:  # two calls in a row
        assert _compare(nctx, step.plan, a, b, step.c) <= TOL


def test_noalloc_refuses_plans_larger_than_its_scratch(nctx):
    from paper_2508_10076_gb300 import api
    V = {q: 100 for q in (-1, 0, 1)}
    s = nctx.space("U1", V)
    A = nctx.tmap([s, s], [s])
    B = nctx.tmap([s], [s, s])
    plan = api.contract_plan(nctx, A, (0,), (1, 2), B, (1, 0), (2,), (0,), (1,))
    assert plan.workspace_bytes > api.NOALLOC_SCRATCH_BYTES
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
