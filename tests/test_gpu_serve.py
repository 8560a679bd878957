"""The continuous-batching request loop: every result served in the mix equals the same request
run alone with tk_contract (bit for bit: the packed launches keep each request's arithmetic), and
the loop reports sensible latencies."""

import numpy as np
import pytest

from paper_2508_10076_gb300 import build_library

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gctx():
    assert torch.cuda.is_available()
    build_library()
    from paper_2508_10076_gb300 import api
    ctx = api.Context(0)
    yield ctx
    ctx.sync()


def test_results_same_alone_and_in_the_mix(gctx):
    from paper_2508_10076_gb300 import api
    from paper_2508_10076_gb300.serve import Server, dimension_grid, request_stream
    grid = dimension_grid(64, 512, 6)
    reqs = request_stream(80, seed=5, grid=grid)
    server = Server(gctx, budget_bytes=2 << 30, streams=3, max_batch=16)
    # a rate far above the service rate: requests arrive while others run, so batches form
    lat, summary, outs = server.run(reqs, rate_per_s=2e5, keep_outputs=True)
    assert summary["batches"] < len(reqs)
    assert np.all(lat > 0) and summary["p50_ms"] <= summary["p99_ms"] <= summary["max_ms"]
    for i, r in enumerate(reqs):
        sh = server.shape(r["sym"], r["D"], r["dtype"])
        c = torch.empty(sh.out_numel, dtype=sh.tdt, device="cuda")
        ws = torch.empty(sh.ws_bytes, dtype=torch.uint8, device="cuda")
        api.contract(gctx, sh.serve_plan, sh.a, sh.b, c, ws)
        torch.cuda.synchronize()
        assert torch.equal(outs[i], c), (i, r)


def test_admission_respects_the_memory_budget(gctx):
    """With a budget that holds a single large request, requests still all complete (admitted as
    memory frees up)."""
    from paper_2508_10076_gb300.serve import Server, dimension_grid, request_stream
    grid = dimension_grid(128, 256, 2)
    reqs = request_stream(12, seed=6, grid=grid)
    server = Server(gctx, budget_bytes=1, streams=2)
    for r in reqs:
        server.shape(r["sym"], r["D"], r["dtype"])
    biggest = max(sh.bytes for sh in server.shapes.values())
    server.budget = biggest
    lat, summary, _ = server.run(reqs, rate_per_s=1e6)
    assert summary["requests"] == 12 and np.all(np.isfinite(lat))


def test_split_precision_solo_requests(gctx):
    """With a split mode on the server, large shapes run one by one in split precision: each result
    equals the same request run alone with the split plan, and stays within 1e-10 of FP64."""
    from paper_2508_10076_gb300 import api
    from paper_2508_10076_gb300.serve import Server, calibrated_rate, dimension_grid, request_stream
    grid = dimension_grid(256, 2048, 4)
    reqs = request_stream(24, seed=8, grid=grid)
    server = Server(gctx, budget_bytes=8 << 30, streams=3, split_gemm="ozaki", solo_ms=0.0)
    for r in reqs:
        server.shape(r["sym"], r["D"], r["dtype"])
    calibrated_rate(server, reqs)
    assert any(sh.solo for sh in server.shapes.values())
    lat, summary, outs = server.run(reqs, rate_per_s=1e5, keep_outputs=True)
    assert summary["requests"] == len(reqs) and np.all(lat > 0)
    for i, r in enumerate(reqs):
        sh = server.shape(r["sym"], r["D"], r["dtype"])
        c = torch.empty(sh.out_numel, dtype=sh.tdt, device="cuda")
        ws = torch.empty(sh.ws_bytes, dtype=torch.uint8, device="cuda")
        api.contract(gctx, sh.serve_plan, sh.a, sh.b, c, ws)
        ref = torch.empty_like(c)
        ws64 = torch.empty(max(1, sh.plan.workspace_bytes), dtype=torch.uint8, device="cuda")
        api.contract(gctx, sh.plan, sh.a, sh.b, ref, ws64)
        torch.cuda.synchronize()
        assert torch.equal(outs[i], c), (i, r)
        err = float(torch.linalg.norm(c - ref) / torch.linalg.norm(ref))
        assert err <= 1e-10, (i, r, err)
