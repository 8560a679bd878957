"""tk_plan_autotune: the tuned plan still matches the oracle, stays within the workspace it was
given, and keeps giving the same bits run after run."""

import numpy as np
import pytest

from harness import oracle_heff, rel_frobenius_per_block
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


@pytest.mark.parametrize("gemm,tol", [("fp64", 1e-12), ("ozaki", 1e-10)])
def test_autotuned_chain_matches_oracle(gctx, gemm, tol):
    from paper_2508_10076_gb300.chain import HeffChain
    ch = HeffChain(gctx, "U1", 1024, gemm=gemm, seed=4)
    limits = [s.plan.workspace_bytes for s in ch.steps]
    choices = ch.autotune()
    assert len(choices) == 4
    for s, lim in zip(ch.steps, limits):
        assert s.plan.workspace_bytes <= 2 * lim
    refs = oracle_heff("U1", 1024, seed=4, tier="block")
    t = ch.steps[0].run(ch.dev["L"], ch.dev["x"])
    outs = [t.clone()]
    for i, other in ((1, "W"), (2, "W"), (3, "R")):
        t = ch.steps[i].run(t, ch.dev[other])
        outs.append(t.clone())
    again = ch.run().clone()
    gctx.sync()
    assert torch.equal(again, outs[-1])
    for i, ((cs, rd), b) in enumerate(zip(refs, outs)):
        assert rel_frobenius_per_block(cs, b.cpu().numpy(), rd) <= tol, i


def test_autotune_respects_the_workspace_it_is_given(gctx):
    from paper_2508_10076_gb300 import api
    from paper_2508_10076_gb300.chain import LxContraction
    lx = LxContraction(gctx, "SU2", 256)
    exact = torch.empty(max(1, lx.step.plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    api.autotune(gctx, lx.step.plan, lx.dev["L"], lx.dev["x"], lx.step.c, exact)
    assert lx.step.plan.workspace_bytes <= exact.numel()
    ref = lx.run().clone()
    gctx.sync()
    assert np.isfinite(ref.cpu().numpy()).all()
