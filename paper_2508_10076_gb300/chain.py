"""Workload drivers over libtk: the two-site effective-Hamiltonian chain x' = L.x.W.W.R
(Algorithm 12 of the paper, repeated application), single L.x contractions and the small C0
contraction.  Everything on the path is a libtk launch; this module allocates device memory
with PyTorch, fills inputs from :mod:`.workloads` and sequences the ABI calls.
"""

import time

import numpy as np
import torch

from . import api
from . import workloads as wl


def _tmap(ctx, sym, legs):
    cod, dom = legs
    return ctx.tmap([ctx.space(sym, s, d) for s, d in cod], [ctx.space(sym, s, d) for s, d in dom])


def mpo_data(tm, entries, numel):
    """Reduced data of the U(1) XXZ MPO in tm's layout (abelian: entries placed by label)."""
    data = np.zeros(numel)
    lookup = {}
    for (wl_q, wl_k), sp, s, (wr_q, wr_k), v in entries:
        lookup[(wl_q, sp, s, wr_q, wl_k, wr_k)] = v
    for unc, si, c, fi, off, ld, dims in tm.treepairs():
        wl_q, sp, s, wr_q = unc
        for kl in range(dims[0]):
            for kr in range(dims[3]):
                v = lookup.get((wl_q, sp, s, wr_q, kl, kr))
                if v is not None:
                    data[off + kl + kr * ld] = v
    return data


def capture_graph(ctx, fn):
    """Record fn() (a sequence of libtk launches on the current stream) into a CUDA graph.

    Two eager runs on a side stream first settle every one-time set-up (plan tables, kernel
    attributes), so the capture contains kernel launches only."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    n0 = ctx.launches
    with torch.cuda.graph(graph):
        out = fn()
    return graph, out, ctx.launches - n0


class Contraction:
    """One planned contraction with its device buffers (inputs, output, workspace)."""

    def __init__(self, ctx, a, b, spec, dtype="f64", gemm="fp64", slices=0, device="cuda"):
        pa, qa, pb, qb, pab, qab = spec
        self.ctx, self.a, self.b = ctx, a, b
        self.plan = api.contract_plan(ctx, a, pa, qa, b, pb, qb, pab, qab, dtype=dtype, gemm=gemm,
                                      slices=slices)
        self.out = self.plan.output()
        tdt = torch.complex128 if dtype == "c128" else torch.float64
        self.c = torch.empty(self.out.numel, dtype=tdt, device=device)
        self.ws = torch.empty(max(1, self.plan.workspace_bytes), dtype=torch.uint8, device=device)

    def run(self, a_buf, b_buf, stream=None):
        api.contract(self.ctx, self.plan, a_buf, b_buf, self.c, self.ws, stream)
        return self.c

    def autotune(self, a_buf, b_buf, headroom=2.0):
        """Let libtk time this contraction's candidate work lists on these operands; the workspace
        may grow up to `headroom` times its heuristic size and is re-sized to the choice."""
        big = torch.empty(max(1, int(self.plan.workspace_bytes * headroom)), dtype=torch.uint8,
                          device=self.ws.device)
        choice = api.autotune(self.ctx, self.plan, a_buf, b_buf, self.c, big)
        self.ws = torch.empty(max(1, self.plan.workspace_bytes), dtype=torch.uint8, device=self.ws.device)
        return choice


class HeffChain:
    """Two-site x' = (((L x) W) W) R (Algorithm 12), or with sites=1 the single-site
    x' = ((L x) W) R (Algorithm 11), with all intermediates resident on the device."""

    def __init__(self, ctx, sym="U1", D=1024, gemm="fp64", slices=0, seed=0, device="cuda",
                 dtype="f64", sites=2, mpo=None):
        self.ctx, self.sym, self.D, self.sites = ctx, sym, D, sites
        V, P, W = wl.heff_spaces(sym, D)
        self.sectors = (V, P, W)
        legs = wl.heff_legs(V, P, W) if sites == 2 else wl.heff1_legs(V, P, W)
        self.legs = legs
        t0 = time.perf_counter()  # structures (spaces, fusion trees, block layout) of the operands
        self.tm = {k: _tmap(ctx, sym, legs[k]) for k in ("x", "L", "W", "R")}
        struct_ms = (time.perf_counter() - t0) * 1e3
        self.host = {}
        rnd = wl.normal_complex if dtype == "c128" else wl.normal
        for i, k in enumerate(("x", "L", "R")):
            self.host[k] = rnd(seed * 16 + i, self.tm[k].numel)
        if sym == "U1":
            w = mpo_data(self.tm["W"], wl.xxz_mpo_entries(), self.tm["W"].numel)
            self.host["W"] = w.astype(np.complex128) if dtype == "c128" else w
        elif mpo == "heisenberg":  # SU(2) Heisenberg MPO (stored reduced entries)
            if sym != "SU2" or self.tm["W"].numel != len(wl.HEISENBERG_SU2_MPO):
                raise ValueError("the Heisenberg MPO is defined for the SU(2) workload spaces")
            w = np.array(wl.HEISENBERG_SU2_MPO, dtype=np.float64)
            self.host["W"] = w.astype(np.complex128) if dtype == "c128" else w
        else:
            self.host["W"] = rnd(seed * 16 + 3, self.tm["W"].numel)
        tdt = torch.complex128 if dtype == "c128" else torch.float64
        self.dev = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device=device, dtype=tdt)
                    for k, v in self.host.items()}
        specs = wl.HEFF_SPECS if sites == 2 else wl.HEFF1_SPECS
        self.others = ("L", "W", "W", "R") if sites == 2 else ("L", "W", "R")
        self.steps = []
        cur = self.tm["x"]
        t0 = time.perf_counter()  # and every contraction plan (the inputs are drawn in between)
        for i, other in enumerate(self.others):
            first = i == 0
            if first:  # T1 = L x : A = L, B = x
                st = Contraction(ctx, self.tm["L"], cur, specs[0], dtype, gemm, slices, device)
            else:
                st = Contraction(ctx, cur, self.tm[other], specs[i], dtype, gemm, slices, device)
            self.steps.append(st)
            cur = st.out
        self.plan_build_ms = struct_ms + (time.perf_counter() - t0) * 1e3
        self.flops = sum(s.plan.flops for s in self.steps)
        self.tensor_flops = sum(s.plan.tensor_flops for s in self.steps)
        self.permute_bytes = sum(s.plan.permute_bytes for s in self.steps)

    def run(self, x=None, stream=None):
        x = self.dev["x"] if x is None else x
        t = self.steps[0].run(self.dev["L"], x, stream)
        for st, other in zip(self.steps[1:], self.others[1:]):
            t = st.run(t, self.dev[other], stream)
        return t

    def run_host(self, host, host_out):
        """One application from pinned host buffers to a pinned host result, every copy through
        the C ABI: x and L are copied and L x runs on the current stream while W and R are copied
        on a side stream (they are needed only by the later steps); x' is read back at the end.
        host: dict of pinned CPU tensors "x", "L", "W", "R" matching the device inputs."""
        main = torch.cuda.current_stream()
        if not hasattr(self, "_copy_stream"):
            self._copy_stream = torch.cuda.Stream(device=self.dev["x"].device)
        side = self._copy_stream

        def h2d(k, st):
            api.copy_h2d(self.ctx, self.dev[k], host[k].data_ptr(), host[k].numel() * host[k].element_size(), st)

        side.wait_stream(main)  # fork: the device copies of W and R are free to overwrite
        h2d("W", side)
        h2d("R", side)
        h2d("x", main)
        h2d("L", main)
        t = self.steps[0].run(self.dev["L"], self.dev["x"], main)
        main.wait_stream(side)  # join before W is read
        for st, other in zip(self.steps[1:], self.others[1:]):
            t = st.run(t, self.dev[other], main)
        api.copy_d2h(self.ctx, host_out.data_ptr(), t, host_out.numel() * host_out.element_size(), main)
        return host_out

    def autotune(self):
        """Tune every step on the chain's own intermediates (before any graph capture)."""
        x = self.dev["x"]
        self.steps[0].run(self.dev["L"], x)
        choices = [self.steps[0].autotune(self.dev["L"], x)]
        for i in range(1, len(self.steps)):
            t, other = self.steps[i - 1].c, self.dev[self.others[i]]
            choices.append(self.steps[i].autotune(t, other))
            self.steps[i].run(t, other)
        return choices

    def capture(self):
        """One application recorded as a CUDA graph: (graph, output buffer, launches per replay)."""
        return capture_graph(self.ctx, self.run)


class LxContraction:
    """T = L x, the environment applied to the two-site tensor (SU(2) workloads)."""

    def __init__(self, ctx, sym="SU2", D=256, gemm="fp64", slices=0, seed=0, device="cuda",
                 dtype="f64"):
        V, P, W = wl.heff_spaces(sym, D)
        legs = wl.heff_legs(V, P, W)
        self.legs = legs
        self.tm = {k: _tmap(ctx, sym, legs[k]) for k in ("x", "L")}
        rnd = wl.normal_complex if dtype == "c128" else wl.normal
        self.host = {"x": rnd(seed * 16 + 0, self.tm["x"].numel), "L": rnd(seed * 16 + 1, self.tm["L"].numel)}
        tdt = torch.complex128 if dtype == "c128" else torch.float64
        self.dev = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device=device, dtype=tdt)
                    for k, v in self.host.items()}
        self.step = Contraction(ctx, self.tm["L"], self.tm["x"], wl.LX_SPEC, dtype, gemm, slices, device)
        self.flops = self.step.plan.flops
        self.tensor_flops = self.step.plan.tensor_flops
        self.permute_bytes = self.step.plan.permute_bytes

    def run(self, stream=None):
        return self.step.run(self.dev["L"], self.dev["x"], stream)

    def autotune(self):
        return [self.step.autotune(self.dev["L"], self.dev["x"])]

    def capture(self):
        return capture_graph(self.step.ctx, self.run)
