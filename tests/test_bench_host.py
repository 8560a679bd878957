"""Host logic of bench.py: the reference arm counts block flops on the oracle's own structures
(it loads no libtk), and that count equals the library planner's for every benched workload."""

import importlib.util
import os

import pytest

from paper_2508_10076_gb300 import api, build_library
from paper_2508_10076_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _library_flops(ctx, name):
    cfg = wl.CONFIGS[name]
    V, P, W = wl.heff_spaces(cfg["sym"], cfg["D"])
    legs = wl.heff1_legs(V, P, W) if cfg["kind"] == "heff1" else wl.heff_legs(V, P, W)

    def tm(k):
        cod, dom = legs[k]
        return ctx.tmap([ctx.space(cfg["sym"], s, d) for s, d in cod], [ctx.space(cfg["sym"], s, d) for s, d in dom])

    if cfg["kind"] == "lx":
        return api.contract_plan(ctx, tm("L"), *wl.LX_SPEC[:2], tm("x"), *wl.LX_SPEC[2:]).flops
    specs = wl.HEFF_SPECS if cfg["kind"] == "heff" else wl.HEFF1_SPECS
    others = ("L", "W", "W", "R") if cfg["kind"] == "heff" else ("L", "W", "R")
    total, cur = 0.0, tm("x")
    for i, spec in enumerate(specs):
        pl = (api.contract_plan(ctx, tm("L"), *spec[:2], cur, *spec[2:]) if i == 0 else
              api.contract_plan(ctx, cur, *spec[:2], tm(others[i]), *spec[2:]))
        total += pl.flops
        cur = pl.output()
    return total


@pytest.mark.parametrize("name", ["c1_u1_heff_d1024", "c3_u1_heff_d4096", "c3_su2_lx_n1024",
                                  "c5_su2_heff1_n1024", "c6_u1su2_heff_n2048"])
def test_oracle_block_flops_equal_the_planners(name):
    build_library()
    bench = _bench()
    assert bench.oracle_block_flops(name) == _library_flops(api.Context(-1), name)


def test_reference_arm_imports_no_library():
    """The reference arm's flop count and oracle runs import nothing that loads libtk."""
    import subprocess
    import sys
    code = ("import sys, importlib.util; sys.path.insert(0, %r); "
            "spec = importlib.util.spec_from_file_location('b', %r); b = importlib.util.module_from_spec(spec); "
            "spec.loader.exec_module(b); b.oracle_block_flops('c1_u1_heff_d1024'); "
            "import paper_2508_10076_gb300._abi as a; assert a._LIB is None, 'libtk was loaded'; "
            "assert not any('libtk' in l for l in open('/proc/self/maps')), 'libtk mapped'") % (ROOT, os.path.join(ROOT, "bench.py"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
