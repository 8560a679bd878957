"""The continuous-batching request loop: every result served in the mix equals the same request
run alone with tk_contract (bit for bit: the packed launches keep each request's arithmetic) and
matches the oracle's contraction of that request (Algorithm 8), admission follows the context's
HBM budget (resident inputs, plan tables, in-flight outputs and workspaces), and the loop reports
sensible latencies."""

import numpy as np
import pytest

from harness import ostruct, rel_frobenius_per_block
from oracle import ops
from paper_2508_10076_gb300 import build_library
from paper_2508_10076_gb300 import workloads as wl

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


_ORACLE = {}


def _oracle_result(ctx, r):
    """(structure, data) of the oracle's L.x for request r's shape, from the same seeded inputs."""
    from paper_2508_10076_gb300.serve import shape_inputs
    key = (r["sym"], r["D"], r["dtype"])
    if key not in _ORACLE:
        legs, _, _, a, b = shape_inputs(ctx, *key)
        _ORACLE[key] = ops.contract(ostruct(r["sym"], legs["L"]), a, *wl.LX_SPEC[:2], ostruct(r["sym"], legs["x"]), b,
                                    *wl.LX_SPEC[2:], tier="block")
    return _ORACLE[key]


def test_results_same_alone_and_in_the_mix(gctx):
    from paper_2508_10076_gb300 import api
    from paper_2508_10076_gb300.serve import Server, dimension_grid, request_stream
    grid = dimension_grid(64, 512, 6)
    reqs = request_stream(80, seed=5, grid=grid)
    before = gctx.memory()["reserved_bytes"]
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
        cs, ref = _oracle_result(gctx, r)
        assert rel_frobenius_per_block(cs, outs[i].cpu().numpy(), ref) <= 1e-12, (i, r)
    assert gctx.memory()["reserved_bytes"] == before + sum(sh.resident for sh in server.shapes.values())
    server.close()
    assert gctx.memory()["reserved_bytes"] == before


def test_admission_respects_the_memory_budget(gctx):
    """The budget counts the plan tables libtk holds and the shapes' resident inputs; with room left
    for a single request beyond those, requests still all complete (admitted one at a time as
    memory frees up), and a budget that cannot hold one request is reported, not waited on."""
    from paper_2508_10076_gb300.serve import Server, dimension_grid, request_stream
    grid = dimension_grid(128, 256, 2)
    reqs = request_stream(12, seed=6, grid=grid)
    server = Server(gctx, budget_bytes=0, streams=2)
    for r in reqs:
        server.shape(r["sym"], r["D"], r["dtype"])
    mem = gctx.memory()
    assert mem["reserved_bytes"] >= sum(sh.resident for sh in server.shapes.values())
    biggest = max(sh.bytes for sh in server.shapes.values())
    server.budget = mem["library_bytes"] + mem["reserved_bytes"] + biggest
    lat, summary, _ = server.run(reqs, rate_per_s=1e6)
    assert summary["requests"] == 12 and np.all(np.isfinite(lat))
    assert gctx.memory()["reserved_bytes"] == mem["reserved_bytes"]  # every admission released
    server.budget = mem["library_bytes"] + mem["reserved_bytes"] + biggest // 2
    with pytest.raises(RuntimeError):
        server.run(reqs, rate_per_s=1e6)
    server.budget = 0
    server.close()


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
        cs, oref = _oracle_result(gctx, r)
        assert rel_frobenius_per_block(cs, outs[i].cpu().numpy(), oref) <= (1e-10 if sh.solo else 1e-12), (i, r)
    server.close()
