"""Failure detection without a GPU fault: a bounded device-side wait that runs out is reported as
TK_ERR_TIMEOUT by the next tk_ctx_sync, the status word is cleared, and the same context keeps
computing correct results.  The wait is on an mbarrier that nothing completes (the kernel
launched by tk_ctx_selftest_timeout); nothing faults, traps or hangs."""

import time

import numpy as np
import pytest

from paper_2508_10076_gb300 import build_library

TK_ERR_TIMEOUT = 8
TK_ERR_NO_DEVICE = 10


def test_selftest_on_host_only_context_is_refused():
    build_library()
    from paper_2508_10076_gb300 import api
    ctx = api.Context(-1)
    with pytest.raises(api.TKError) as e:
        ctx.selftest_timeout()
    assert e.value.code == TK_ERR_NO_DEVICE


@pytest.mark.gpu
def test_bounded_wait_times_out_and_context_stays_usable():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    build_library()
    from paper_2508_10076_gb300 import api
    ctx = api.Context(0)
    ctx.sync()
    t0 = time.perf_counter()
    ctx.selftest_timeout()
    with pytest.raises(api.TKError) as e:
        ctx.sync()
    waited = time.perf_counter() - t0
    assert e.value.code == TK_ERR_TIMEOUT
    assert "kernel tag 9" in str(e.value)
    assert 1.5 < waited < 60.0, waited  # the device-side limit is 2 s
    ctx.sync()  # the status word was cleared by the report

    # the same context still runs the split-precision pipeline (bounded waits on every stage)
    V = ctx.space("U1", {-2: 30, -1: 70, 0: 150, 1: 70, 2: 30})
    P = ctx.space("U1", {-1: 1, 1: 1})
    A = ctx.tmap([V, P], [V])
    B = ctx.tmap([V], [V, P])
    gen = np.random.default_rng(11)
    a = torch.from_numpy(gen.standard_normal(A.numel)).cuda()
    b = torch.from_numpy(gen.standard_normal(B.numel)).cuda()
    out = {}
    for gemm in ("fp64", "ozaki"):
        plan = api.compose_plan(ctx, A, B, gemm=gemm)
        c = torch.empty(plan.output().numel, dtype=torch.float64, device="cuda")
        ws = torch.empty(max(plan.workspace_bytes, 1), dtype=torch.uint8, device="cuda")
        api.contract(ctx, plan, a, b, c, ws)
        ctx.sync()
        out[gemm] = c
    rel = (torch.linalg.norm(out["ozaki"] - out["fp64"]) / torch.linalg.norm(out["fp64"])).item()
    assert rel < 1e-10, rel
