"""Continuous-batching request loop over libtk (C4 serving workload; the paper has no serving
layer).  Requests are single contractions L.x of the two-site effective Hamiltonian (U(1) at bond
dimension D, SU(2) at reduced multiplicity D/4), FP64 or complex128, arriving as a Poisson stream.

Scheduling, per pass of the loop:
  * requests whose arrival time has passed join the queue;
  * the HBM budget is the context's (tk_ctx_set_budget): the plan tables libtk holds count against
    it, every shape's resident inputs are reserved when the shape is created (tk_ctx_reserve), and a
    queued request is admitted while its output + workspace can be reserved too (TK_ERR_BUDGET
    otherwise) and an in-flight slot is free; a finished batch releases its reservation;
  * the admitted requests of one dtype go to the GPU together through tk_contract_batch (their
    permutes, zero fills and sector-GEMM tiles share launches) on the next of several CUDA streams,
    so batches overlap on the device while new requests keep arriving;
  * optionally (split_gemm), shapes whose FP64 service time alone is at least solo_ms and whose
    split-precision time is shorter run one by one in that mode (Ozaki BF16: within 1e-10 of FP64)
    instead of in the FP64 batches;
  * finished batches (their end event has completed) release memory and slots.
Latency = completion time on the device clock - arrival time, both relative to one start event.
Plans (structure, recoupling tables, GEMM work lists) are built once per shape, autotuned once
on the shape's resident inputs (tk_plan_autotune) before any request is timed, and stay resident.
"""

import time

import numpy as np
import torch

from . import api
from . import workloads as wl


def _tmap(ctx, sym, legs):
    cod, dom = legs
    return ctx.tmap([ctx.space(sym, s, d) for s, d in cod], [ctx.space(sym, s, d) for s, d in dom])


def dimension_grid(lo=64, hi=4096, levels=25):
    """Bond dimensions on a geometric grid: a log-uniform draw is rounded to the nearest level, so
    that the plan cache sees a bounded set of shapes."""
    return sorted({int(round(lo * (hi / lo) ** (i / (levels - 1)))) for i in range(levels)})


def request_stream(n, seed=0, rate_per_s=None, grid=None):
    """n requests (arrival_s, sym, D, dtype): symmetry 1:1 U(1)/SU(2), dtype 1:1 float64/complex128,
    D log-uniform on [64, 4096] rounded to `grid`, Poisson arrivals at rate_per_s (filled in by the
    caller when None)."""
    rng = np.random.default_rng(seed)
    grid = np.array(grid or dimension_grid())
    logd = rng.uniform(np.log(grid[0]), np.log(grid[-1]), n)
    D = grid[np.abs(np.log(grid)[None, :] - logd[:, None]).argmin(axis=1)]
    sym = np.where(rng.random(n) < 0.5, "U1", "SU2")
    dtype = np.where(rng.random(n) < 0.5, "f64", "c128")
    gaps = rng.exponential(1.0, n)  # unit-rate Poisson gaps, scaled by 1/rate later
    return [dict(idx=i, gap=float(gaps[i]), sym=str(sym[i]), D=int(D[i]), dtype=str(dtype[i])) for i in range(n)]


def shape_inputs(ctx, sym, D, dtype, seed=0):
    """(legs, L structure, x structure, host data of L, host data of x) of one request shape: U(1)
    at bond dimension D, SU(2) at reduced multiplicity D/4 (at least 8), seeded N(0,1) blocks
    (N(0,1/2) per component for complex128)."""
    V, P, W = wl.heff_spaces(sym, D if sym == "U1" else max(8, D // 4))
    legs = wl.heff_legs(V, P, W)
    L, x = _tmap(ctx, sym, legs["L"]), _tmap(ctx, sym, legs["x"])
    rnd = wl.normal_complex if dtype == "c128" else wl.normal
    return legs, L, x, np.ascontiguousarray(rnd(seed * 16 + 1, L.numel)), np.ascontiguousarray(rnd(seed * 16 + 0, x.numel))


class Shape:
    """Plans and resident inputs of one request shape (symmetry, D, dtype).  The resident inputs
    are reserved against the context's budget for the life of the shape."""

    def __init__(self, ctx, sym, D, dtype, seed=0, split_gemm=None):
        legs, L, x, a_host, b_host = shape_inputs(ctx, sym, D, dtype, seed)
        self.legs = legs
        self.plan = api.contract_plan(ctx, L, *wl.LX_SPEC[:2], x, *wl.LX_SPEC[2:], dtype=dtype)
        self.flops = self.plan.flops
        self.tdt = torch.complex128 if dtype == "c128" else torch.float64
        self.esize = 16 if dtype == "c128" else 8
        self.resident = (L.numel + x.numel) * self.esize
        ctx.reserve(self.resident)
        self.a = torch.from_numpy(a_host).to("cuda", self.tdt)
        self.b = torch.from_numpy(b_host).to("cuda", self.tdt)
        self.split_plan = (api.contract_plan(ctx, L, *wl.LX_SPEC[:2], x, *wl.LX_SPEC[2:], dtype=dtype, gemm=split_gemm)
                           if split_gemm else None)
        self.solo = False  # served alone in split precision (set by calibrated_rate)
        self.out_numel = self.plan.output().numel
        self.tuned = False

    def autotune(self, ctx):
        """Pick each plan's work list on the resident inputs (tk_plan_autotune), once."""
        if self.tuned:
            return
        for plan in (self.plan, self.split_plan):
            if plan is None:
                continue
            c = torch.empty(self.out_numel, dtype=self.tdt, device="cuda")
            ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
            api.autotune(ctx, plan, self.a, self.b, c, ws)
        self.tuned = True

    @property
    def serve_plan(self):
        return self.split_plan if self.solo else self.plan

    @property
    def ws_bytes(self):
        return max(1, self.serve_plan.workspace_bytes)

    @property
    def bytes(self):
        """Device bytes of one request in flight: its output and its workspace."""
        return self.out_numel * self.esize + self.ws_bytes


class Server:
    def __init__(self, ctx, budget_bytes=150 << 30, streams=3, max_batch=64, max_inflight=256,
                 split_gemm=None, solo_ms=1.0, autotune=True):
        self.ctx = ctx
        self.split_gemm = split_gemm
        self.solo_ms = solo_ms
        self.budget = budget_bytes
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.max_batch = max_batch
        self.max_inflight = max_inflight
        self.autotune = autotune
        self.shapes = {}

    @property
    def budget(self):
        return self.ctx.memory()["budget_bytes"]

    @budget.setter
    def budget(self, nbytes):
        """The HBM budget of the server's context (tk_ctx_set_budget)."""
        self.ctx.set_budget(int(nbytes))

    def shape(self, sym, D, dtype):
        key = (sym, D, dtype)
        if key not in self.shapes:
            sh = Shape(self.ctx, sym, D, dtype, split_gemm=self.split_gemm)
            if self.autotune:
                sh.autotune(self.ctx)
            self.shapes[key] = sh
        return self.shapes[key]

    def close(self):
        """Drop the shapes: their resident inputs' reservations go back to the context."""
        for sh in self.shapes.values():
            self.ctx.release(sh.resident)
        self.shapes = {}

    def _admit(self, nbytes):
        """Reserve a request's output + workspace against the budget; False if it does not fit."""
        try:
            self.ctx.reserve(nbytes)
            return True
        except api.TKError as e:
            if e.code != 11:  # TK_ERR_BUDGET
                raise
            return False

    def run(self, requests, rate_per_s, keep_outputs=False):
        """Serve `requests` (from request_stream) arriving at rate_per_s; returns per-request
        latencies (ms) and summary figures.  keep_outputs keeps every result for checking."""
        for r in requests:  # plans and resident inputs first: no plan building inside the timed loop
            self.shape(r["sym"], r["D"], r["dtype"])
        arrivals = np.cumsum([r["gap"] for r in requests]) / rate_per_s
        torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_start.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        host0 = time.perf_counter()
        pending = list(range(len(requests)))  # in arrival order
        queue, inflight, done = [], [], {}
        slots, next_stream, p = 0, 0, 0
        outputs = {}
        batches = 0
        while p < len(pending) or queue or inflight:
            now = time.perf_counter() - host0
            while p < len(pending) and arrivals[pending[p]] <= now:
                queue.append(pending[p])
                p += 1
            # retire finished batches
            still = []
            for b in inflight:
                if b["end"].query():
                    t_end = t_start.elapsed_time(b["end"])  # ms since start, device clock
                    for i in b["reqs"]:
                        done[i] = t_end - 1e3 * arrivals[i]
                    self.ctx.release(b["bytes"])
                    slots -= len(b["reqs"])
                    if not keep_outputs:
                        b["bufs"] = None
                else:
                    still.append(b)
            inflight = still
            # admit and launch: one FP64 batch per dtype, split-precision requests one by one
            admitted = {"f64": [], "c128": []}
            solo = []
            rest = []
            for i in queue:
                r = requests[i]
                sh = self.shape(r["sym"], r["D"], r["dtype"])
                group = solo if sh.solo else admitted[r["dtype"]]
                if (slots < self.max_inflight and (sh.solo or len(group) < self.max_batch) and
                        self._admit(sh.bytes)):
                    group.append(i)
                    slots += 1
                else:
                    rest.append(i)
            queue = rest
            if queue and not inflight and slots == 0:
                r = requests[queue[0]]
                raise RuntimeError(f"request {r} needs {self.shape(r['sym'], r['D'], r['dtype']).bytes} bytes, more "
                                   f"than the budget leaves with nothing in flight ({self.ctx.memory()})")
            for dt, group in admitted.items():
                if not group:
                    continue
                stream = self.streams[next_stream % len(self.streams)]
                next_stream += 1
                with torch.cuda.stream(stream):
                    shapes = [self.shape(requests[i]["sym"], requests[i]["D"], dt) for i in group]
                    outs = [torch.empty(sh.out_numel, dtype=sh.tdt, device="cuda") for sh in shapes]
                    wss = [torch.empty(sh.ws_bytes, dtype=torch.uint8, device="cuda") for sh in shapes]
                    api.contract_batch(self.ctx, [sh.plan for sh in shapes], [sh.a for sh in shapes],
                                       [sh.b for sh in shapes], outs, wss, stream)
                    end = torch.cuda.Event(enable_timing=True)
                    end.record(stream)
                batches += 1
                inflight.append(dict(reqs=group, end=end, bytes=sum(sh.bytes for sh in shapes),
                                     bufs=(outs, wss)))
                if keep_outputs:
                    for i, o in zip(group, outs):
                        outputs[i] = o
            for i in solo:
                r = requests[i]
                sh = self.shape(r["sym"], r["D"], r["dtype"])
                stream = self.streams[next_stream % len(self.streams)]
                next_stream += 1
                with torch.cuda.stream(stream):
                    out = torch.empty(sh.out_numel, dtype=sh.tdt, device="cuda")
                    ws = torch.empty(sh.ws_bytes, dtype=torch.uint8, device="cuda")
                    api.contract(self.ctx, sh.split_plan, sh.a, sh.b, out, ws, stream)
                    end = torch.cuda.Event(enable_timing=True)
                    end.record(stream)
                batches += 1
                inflight.append(dict(reqs=[i], end=end, bytes=sh.bytes, bufs=(out, ws)))
                if keep_outputs:
                    outputs[i] = out
            if not admitted["f64"] and not admitted["c128"] and not solo:
                time.sleep(20e-6)  # nothing to launch: wait for arrivals or completions
        torch.cuda.synchronize()
        lat = np.array([done[i] for i in range(len(requests))])
        flops = sum(self.shape(r["sym"], r["D"], r["dtype"]).flops for r in requests)
        # from the first arrival to the last completion, on the device clock
        makespan = max(float(np.max(lat + 1e3 * arrivals)) - 1e3 * float(arrivals[0]), 1e-9)
        summary = {
            "requests": len(requests), "batches": batches, "rate_per_s": rate_per_s,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "throughput_req_per_s": len(requests) / (makespan * 1e-3),
            "block_gflops": flops / (makespan * 1e-3) / 1e9,
            "makespan_ms": makespan,
        }
        return lat, summary, outputs


def _alone_time(server, sh, plan):
    c = torch.empty(sh.out_numel, dtype=sh.tdt, device="cuda")
    ws = torch.empty(max(1, plan.workspace_bytes), dtype=torch.uint8, device="cuda")
    api.contract(server.ctx, plan, sh.a, sh.b, c, ws)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(3):
        api.contract(server.ctx, plan, sh.a, sh.b, c, ws)
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / 3 * 1e-3


def calibrated_rate(server, requests, load=0.7):
    """Arrival rate that keeps the GPU about `load` busy: each shape's service time is measured
    once with tk_contract on its own, and the rate is load / mean service time.  With a split mode
    on the server, a shape is served alone in that mode when its FP64 time is at least solo_ms and
    the split-precision time is shorter."""
    times = {}
    for key, sh in server.shapes.items():
        t64 = _alone_time(server, sh, sh.plan)
        times[key] = t64
        if sh.split_plan is not None and t64 * 1e3 >= server.solo_ms:
            ts = _alone_time(server, sh, sh.split_plan)
            if ts < t64:
                sh.solo = True
                times[key] = ts
    mean = float(np.mean([times[(r["sym"], r["D"], r["dtype"])] for r in requests]))
    return load / mean, mean


