"""Tensor maps without elements on the GPU.  A map whose codomain and domain share no coupled
sector has no blocks (Sec. 3: blocks exist only for coupled sectors admissible on both sides), and
PyTorch hands out NULL for its empty buffers.  Calls on such maps succeed; a call whose output has
no elements launches nothing; a contraction of empty operands into a non-empty output writes the
zero blocks (K_c = 0), as the oracle does."""

import numpy as np
import pytest

from harness import ostruct
from oracle import ops
from paper_2508_10076_gb300 import build_library

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LEGS = {  # U(1): t : V1 (x) V2 <- W is empty (charge 2 against 0); u : V1 (x) V2 <- X is not
    "V1": {1: 2}, "V2": {1: 3}, "W": {0: 1}, "X": {2: 4}, "Y": {5: 2},
}


def _maps(ctx):
    sp = {k: ctx.space("U1", v) for k, v in LEGS.items()}
    return {
        "t": ctx.tmap([sp["V1"], sp["V2"]], [sp["W"]]),    # 0 elements
        "b": ctx.tmap([sp["W"]], [sp["X"]]),                # 0 elements
        "by": ctx.tmap([sp["W"]], [sp["Y"]]),               # 0 elements
    }


def _olegs(cod, dom):
    return ostruct("U1", ([(LEGS[k], False) for k in cod], [(LEGS[k], False) for k in dom]))


def _dt(dtype):
    return torch.complex128 if dtype == "c128" else torch.float64


@pytest.mark.parametrize("dtype", ["f64", "c128"])
def test_permute_and_svd_of_an_empty_map_launch_nothing(dtype):
    build_library()
    from paper_2508_10076_gb300 import api
    ctx = api.Context(0)
    m = _maps(ctx)
    assert m["t"].numel == 0
    empty = torch.empty(0, dtype=_dt(dtype), device="cuda")
    n0 = ctx.launches
    p = api.permute_plan(ctx, m["t"], (2, 1), (0,), dtype=dtype)
    assert p.output().numel == 0
    api.permute(ctx, p, empty, empty)
    api.permute(ctx, p, None, None)
    sp = api.svd_plan(ctx, m["t"], dtype=dtype)
    u, vh, nval = sp.outputs()
    assert u.numel == 0 and vh.numel == 0 and nval == 0 and sp.blocks() == []
    api.svd(ctx, sp, empty, empty, torch.empty(0, dtype=torch.float64, device="cuda"), empty,
            torch.empty(max(1, sp.workspace_bytes), dtype=torch.uint8, device="cuda"))
    api.svd_truncate(ctx, sp, [], None, None, None, None, None, None)
    ctx.sync()
    assert ctx.launches == n0


@pytest.mark.parametrize("dtype,gemm", [("f64", "fp64"), ("f64", "ozaki"), ("f64", "tf32x3"),
                                        ("c128", "fp64"), ("c128", "ozaki")])
def test_contraction_of_empty_operands(dtype, gemm):
    """C = t o b : V1 (x) V2 <- X has one block (24 elements) with K = 0: every call must write its
    zeros over whatever C held, through tk_contract, tk_contract_batch and tk_contract_noalloc.
    C = t o by is empty as a whole: nothing is launched."""
    build_library()
    from paper_2508_10076_gb300 import api
    ctx = api.Context(0)
    m = _maps(ctx)
    tdt = _dt(dtype)
    cs, ref = ops.contract(_olegs(["V1", "V2"], ["W"]), np.zeros(0), (0, 1), (2,),
                           _olegs(["W"], ["X"]), np.zeros(0), (0,), (1,), (0, 1), (2,), tier="block")
    assert cs.numel == 24 and not ref.any()
    plan = api.compose_plan(ctx, m["t"], m["b"], dtype=dtype, gemm=gemm)
    assert plan.output().numel == 24 and plan.flops == 0
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    empty = torch.empty(0, dtype=tdt, device="cuda")
    for run in ("contract", "batch", "noalloc", "autotune"):
        c = torch.full((24,), float("nan"), dtype=tdt, device="cuda")
        if run == "contract":
            api.contract(ctx, plan, empty, empty, c, ws)
        elif run == "batch":
            if dtype == "c128" and gemm != "fp64":
                continue  # complex split-precision plans are not batched
            c2 = torch.full((24,), float("nan"), dtype=tdt, device="cuda")
            ws2 = torch.empty_like(ws)
            api.contract_batch(ctx, [plan, plan], [empty, None], [None, empty], [c, c2], [ws, ws2])
            ctx.sync()
            assert torch.equal(c2.cpu(), torch.zeros(24, dtype=tdt))
        elif run == "noalloc":
            api.contract_noalloc(ctx, plan, None, None, c)
        else:
            api.autotune(ctx, plan, empty, empty, c, ws)
            api.contract(ctx, plan, empty, empty, c, ws)
        ctx.sync()
        got = c.cpu().numpy()
        assert np.array_equal(got, ref.astype(got.dtype)), run
    plan0 = api.compose_plan(ctx, m["t"], m["by"], dtype=dtype, gemm=gemm)
    assert plan0.output().numel == 0
    n0 = ctx.launches
    api.contract(ctx, plan0, None, None, None, torch.empty(max(1, plan0.workspace_bytes), dtype=torch.uint8,
                                                           device="cuda"))
    api.contract_noalloc(ctx, plan0, None, None, None)
    ctx.sync()
    assert ctx.launches == n0
