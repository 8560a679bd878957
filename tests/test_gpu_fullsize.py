"""Parity at the full workload sizes, in the launch configuration the benchmark times: work
lists chosen by the autotuner, one application replayed from a CUDA graph.  Every intermediate is
compared with the oracle's block tier, element by element (relative Frobenius error per block).

Tolerances: FP64 1e-12, Ozaki BF16 (6 slices) 1e-10, 3xTF32 2e-5 (FP32-class; reported, not the
FP64-class bar)."""

import pytest

from harness import oracle_heff, rel_frobenius_per_block
from paper_2508_10076_gb300 import build_library
from paper_2508_10076_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ozaki": 1e-10, "tf32x3": 2e-5}


@pytest.fixture(scope="module")
def gctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build_library()
    from paper_2508_10076_gb300 import api
    ctx = api.Context(0)
    yield ctx
    torch.cuda.synchronize()
    ctx.sync()


def _check_chain(ch, refs, tol):
    ch.autotune()
    graph, _, launches = ch.capture()
    assert launches > 0
    graph.replay()
    torch.cuda.synchronize()
    steps = ch.steps if hasattr(ch, "steps") else [ch.step]
    assert len(steps) == len(refs)
    for i, ((cs, rd), st) in enumerate(zip(refs, steps)):
        assert st.out.blocks() == [(c, r, k, o) for c, r, k, o in cs.blocks], i
        err = rel_frobenius_per_block(cs, st.c.cpu().numpy(), rd)
        assert err <= tol, (i, err)


@pytest.mark.parametrize("gemm", ["fp64", "ozaki", "tf32x3"])
@pytest.mark.parametrize("name", ["c3_u1_heff_d4096", "c5_u1_heff1_d4096", "c6_u1su2_heff_n2048",
                                  "c7_su2_heisenberg_heff_n1024", "c5_su2_heff1_n1024"])
def test_full_size_chain(gctx, name, gemm):
    from paper_2508_10076_gb300.chain import HeffChain
    cfg = wl.CONFIGS[name]
    sites = 2 if cfg["kind"] == "heff" else 1
    ch = HeffChain(gctx, cfg["sym"], cfg["D"], gemm=gemm, sites=sites, mpo=cfg.get("mpo"))
    refs = oracle_heff(cfg["sym"], cfg["D"], tier="block", sites=sites, mpo=cfg.get("mpo"))
    _check_chain(ch, refs, TOL[gemm])


@pytest.mark.parametrize("gemm", ["fp64", "ozaki", "tf32x3"])
def test_full_size_su2_lx(gctx, gemm):
    """C3 SU(2): the environment applied to the two-site tensor at reduced multiplicity 1024."""
    from paper_2508_10076_gb300.chain import LxContraction
    ch = LxContraction(gctx, "SU2", 1024, gemm=gemm)
    refs = oracle_heff("SU2", 1024, tier="block", steps=1)
    _check_chain(ch, refs, TOL[gemm])
