"""Benchmark of the symmetric-contraction hot path on GB300 (one JSON line on rank 0).

Default workload: the U(1) two-site effective-Hamiltonian application x' = L.x.W.W.R at
D = 4096 (charges -16..16, n_q ~ exp(-q^2/72)), XXZ MPO -- four pairwise contractions, each a
fusion-tree permute of both operands, one grouped GEMM over the coupled sectors and the output
permute.  A step is one application of the chain.  `value` is the plain FP64 path; the same line
carries the split-precision paths (Ozaki BF16 slices and 3xTF32 on tcgen05) on the same workload,
the D = 1024 chain and the SU(2) L.x at reduced multiplicity 1024 as extra workloads, and the
serving loop (10,000 mixed requests, p50 / p99).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config NAME] [--gemm fp64|ozaki]

Under torchrun (N > 1) every rank runs its own replica of the workload (independent problems,
no collective on the data path): value = all ranks' block flops / max-over-ranks time.
"""

import argparse
import json
import os
import resource
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "symmetric contraction block-GFLOP/s (FP64 vs split-prec); serve p50/p99 ms"
UNIT = "block-GFLOP/s"
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2
DEFAULT_CONFIG = "c3_u1_heff_d4096"
EXTRA_CONFIGS = ("c1_u1_heff_d1024", "c3_su2_lx_n1024")
# DRAM bytes (read + write) per launch of the FP64 sector GEMM on the D = 4096 U(1) chain: the mean
# over the four launches of one application in the timed region, from one ncu capture of the
# current kernel (None for workloads without a capture).
K2_TRAFFIC_BYTES = {"c3_u1_heff_d4096": 1.856e8}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        self.idx = vis.split(",")[local_rank] if vis else str(local_rank)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.idx, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.strip().splitlines():
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(dist, x):
    """The largest of every rank's x (x itself on a single process)."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(flops_per_step, steps, world, total_ms):
    """Whole-job block-GFLOP/s: every rank runs `steps` steps of its own replica; the job takes as
    long as its slowest rank."""
    return flops_per_step * steps * world / (total_ms * 1e-3) / 1e9


def replica_seed(rank):
    """Each rank draws its own inputs: the replicas are independent problems of the same shape."""
    return rank


def _workload(ctx, name, gemm, dtype="f64", seed=0, slices=0):
    from paper_2508_10076_gb300 import workloads as wl
    from paper_2508_10076_gb300.chain import HeffChain, LxContraction
    cfg = wl.CONFIGS[name]
    if cfg["kind"] in ("heff", "heff1"):
        return HeffChain(ctx, cfg["sym"], cfg["D"], gemm=gemm, dtype=dtype, seed=seed,
                         sites=2 if cfg["kind"] == "heff" else 1, mpo=cfg.get("mpo"), slices=slices)
    if cfg["kind"] == "lx":
        return LxContraction(ctx, cfg["sym"], cfg["D"], gemm=gemm, dtype=dtype, seed=seed, slices=slices)
    raise SystemExit(f"config {name} is a parity case, not a bench line")


def _inputs(work):
    from paper_2508_10076_gb300.chain import HeffChain
    if isinstance(work, HeffChain):
        return [work.dev[k] for k in ("x", "L", "W", "R")]
    return [work.dev[k] for k in ("L", "x")]


def _out_blocks(work):
    return (work.steps[-1].out if hasattr(work, "steps") else work.step.out).blocks()


def rel_err_per_block(blocks, got, ref):
    """Largest per-block relative Frobenius difference (numpy arrays or tensors on the host)."""
    import numpy as np
    got, ref = np.asarray(got), np.asarray(ref)
    total = max(float(np.linalg.norm(ref)), 1e-300)
    worst = 0.0
    for _, r, k, o in blocks:
        d = float(np.linalg.norm(got[o:o + r * k] - ref[o:o + r * k]))
        n = float(np.linalg.norm(ref[o:o + r * k]))
        worst = max(worst, d / (n if n > 1e-13 * total else total))
    return worst


# ------------------------------------------------------------------------------------------ oracle
def _oracle_run(name):
    """A callable running the oracle's block tier on workload `name` (seed 0) and returning its
    result's data."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from harness import oracle_heff, oracle_heff_inputs  # noqa: E402
    from oracle import ops  # noqa: E402
    from paper_2508_10076_gb300 import workloads as wl
    cfg = wl.CONFIGS[name]
    if cfg["kind"] in ("heff", "heff1"):
        sites = 2 if cfg["kind"] == "heff" else 1
        return lambda: oracle_heff(cfg["sym"], cfg["D"], tier="block", sites=sites, mpo=cfg.get("mpo"))[-1][1]
    st, data = oracle_heff_inputs(cfg["sym"], cfg["D"])
    return lambda: ops.contract(st["L"], data["L"], *wl.LX_SPEC[:2], st["x"], data["x"], *wl.LX_SPEC[2:],
                                tier="block")[1]


def oracle_block_flops(name):
    """Block flops of one step of workload `name` counted on the oracle's own structures: sum over
    the coupled sectors of every contraction of 2 M K N, with M, K from the permuted A's block and
    N from the permuted B's block (sectors with K = 0 cost nothing)."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from harness import ostruct  # noqa: E402
    from oracle import TensorStructure  # noqa: E402
    from oracle.ops import permute_spaces  # noqa: E402
    from paper_2508_10076_gb300 import workloads as wl
    cfg = wl.CONFIGS[name]
    V, P, W = wl.heff_spaces(cfg["sym"], cfg["D"])
    legs = wl.heff1_legs(V, P, W) if cfg["kind"] == "heff1" else wl.heff_legs(V, P, W)
    st = {k: ostruct(cfg["sym"], legs[k]) for k in ("x", "L", "W", "R")}

    def one(a, pa, qa, b, pb, qb, pab, qab):
        at = TensorStructure(*permute_spaces(a, pa, qa))
        bt = TensorStructure(*permute_spaces(b, pb, qb))
        bb = {c: (r, k) for c, r, k, _ in bt.blocks}
        flops = 0.0
        for c, m, k, _ in at.blocks:
            if c in bb and k > 0:
                flops += 2.0 * m * k * bb[c][1]
        ct = TensorStructure(at.cod, bt.dom)
        return flops, TensorStructure(*permute_spaces(ct, pab, qab))

    if cfg["kind"] == "lx":
        return one(st["L"], *wl.LX_SPEC[:2], st["x"], *wl.LX_SPEC[2:])[0]
    specs = wl.HEFF_SPECS if cfg["kind"] == "heff" else wl.HEFF1_SPECS
    others = ("L", "W", "W", "R") if cfg["kind"] == "heff" else ("L", "W", "R")
    total, cur = 0.0, st["x"]
    for i, spec in enumerate(specs):
        a, b = (st["L"], cur) if i == 0 else (cur, st[others[i]])
        f, cur = one(a, *spec[:2], b, *spec[2:])
        total += f
    return total


def cpu_baseline(name, budget_s=15.0):
    """The oracle's block tier on the same workload, repeated for a bounded time on the host.
    Returns (applications, wall seconds, effective cores = CPU seconds / wall seconds, BLAS
    threads available, the oracle's result)."""
    run = _oracle_run(name)
    result = run()  # warm caches of the oracle; its result doubles as the error reference
    r0, n, t0 = resource.getrusage(resource.RUSAGE_SELF), 0, time.perf_counter()
    while True:
        run()
        n += 1
        if time.perf_counter() - t0 >= budget_s or n >= 200:
            break
    dt = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    try:
        from threadpoolctl import threadpool_info
        threads = max((i.get("num_threads", 1) for i in threadpool_info()), default=os.cpu_count())
    except Exception:
        threads = os.cpu_count()
    return n, dt, cpu / dt, threads, result


def cpu_baseline_single_thread(name, budget_s):
    """The same oracle run in a fresh process whose BLAS and OpenMP pools hold one thread (the
    paper's own timings are single-threaded); returns (applications, seconds)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
              "NUMEXPR_NUM_THREADS", "VECLIB_MAXIMUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""  # the worker needs no GPU
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", "--config", name,
                        "--cpu-budget", str(budget_s)], env=env, capture_output=True, text=True,
                       timeout=20 * budget_s + 300)
    if r.returncode != 0:
        raise RuntimeError("single-thread CPU baseline failed: " + r.stderr[-500:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return out["n"], out["dt"]


def run_reference(args):
    """The reference arm: the oracle's block tier (the paper's method written out plainly, on the
    host cores), timed on the same workload, metric and unit; no GPU and no libtk."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    flops = oracle_block_flops(args.config)
    per_step = max(1.0, args.budget / max(1, args.steps))
    for _ in range(args.warmup):
        cpu_baseline(args.config, budget_s=0.0)
    times, cores = [], []
    for _ in range(args.steps):
        n, dt, eff, threads, _ = cpu_baseline(args.config, budget_s=per_step)
        times.append(dt / n)
        cores.append(eff)
    ms = 1e3 * statistics.mean(times)
    value = flops / (ms * 1e-3) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.config, "gemm": "fp64 (numpy BLAS)", "tier": "oracle block tier",
                   "block_flops_per_step": flops, "flops_source": "the oracle's own structures"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": round(statistics.mean(cores), 1),
                         "threads_available": threads, "kind": "oracle",
                         "sample": f"whole {args.config} applications repeated for ~{per_step:.0f}s per step; "
                                   "cores = CPU seconds / wall seconds"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------ GPU arm
class Timer:
    """K steps, the L2 flushed before each, CUDA events on the launching stream around each."""

    def __init__(self, torch, stream, flush, barrier):
        self.torch, self.stream, self.flush, self.barrier = torch, stream, flush, barrier

    def __call__(self, fn, steps, clocks=None, label="timed"):
        """Total ms of `steps` timed calls of fn; clocks (a Clocks) samples the timed region only.
        The region is an NVTX range named `label` (ncu --nvtx-include selects its launches)."""
        t = self.torch
        starts = [t.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [t.cuda.Event(enable_timing=True) for _ in range(steps)]
        self.barrier()
        if clocks is not None:
            clocks.start()
        t.cuda.nvtx.range_push(label)
        for i in range(steps):
            self.flush.zero_()
            starts[i].record(self.stream)
            fn()
            ends[i].record(self.stream)
        t.cuda.nvtx.range_pop()
        self.barrier()
        if clocks is not None:
            self.clk = clocks.stop()
        return sum(s.elapsed_time(e) for s, e in zip(starts, ends))


def measure(ctx, name, gemm, args, timer, rank, steps, want_graph=True, clocks=None, slices=0):
    """One workload in one GEMM mode: autotune, warm up, capture one step as a CUDA graph, time
    `steps` replays, then the same loop eager with libtk's launch profiler on."""
    work = _workload(ctx, name, gemm, seed=replica_seed(rank), slices=slices)
    tuned = work.autotune() if not args.no_autotune else None  # before any graph capture
    for _ in range(max(3, args.warmup)):
        work.run()
    ctx.sync()
    step_fn, per_step_launches, mode, graph_out = work.run, None, "eager", None
    if want_graph and not args.eager:
        try:
            graph, graph_out, per_step_launches = work.capture()
            step_fn, mode = graph.replay, "cuda_graph"
            for _ in range(max(3, args.warmup)):
                step_fn()
        except Exception as exc:  # keep the eager path; report why
            step_fn, mode = work.run, f"eager (graph capture failed: {exc})"
    timer.torch.cuda.synchronize()
    launches0 = ctx.launches
    total_ms = timer(step_fn, steps, clocks, label=f"timed_{name}_{gemm}" + (f"_s{slices}" if slices else ""))
    launches = ctx.launches - launches0 if per_step_launches is None else per_step_launches * steps
    ctx.sync()
    ctx.profile(True)
    for _ in range(steps):
        timer.flush.zero_()
        work.run()
    ctx.sync()
    prof = ctx.profile_read()
    ctx.profile(False)
    out = (graph_out if graph_out is not None else work.run())
    timer.torch.cuda.synchronize()
    return dict(work=work, tuned=tuned, step_fn=step_fn, mode=mode, graph_out=graph_out, total_ms=total_ms,
                launches=launches, prof=prof, out=out.clone())


def measure_svd(api, ctx, tm, data, torch, reps=5):
    """The block SVD after the two-site step (Alg. 9 in Alg. 12) of one chain's result x': one
    k_svd_jacobi launch over every coupled sector, timed with CUDA events (median of `reps` after a
    warm-up), its singular values checked block by block against numpy's LAPACK SVD."""
    import numpy as np
    sp = api.svd_plan(ctx, tm)
    u_t, vh_t, nval = sp.outputs()
    u = torch.empty(u_t.numel, dtype=torch.float64, device="cuda")
    vh = torch.empty(vh_t.numel, dtype=torch.float64, device="cuda")
    s = torch.empty(max(1, nval), dtype=torch.float64, device="cuda")
    ws = torch.empty(max(1, sp.workspace_bytes), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    api.svd(ctx, sp, data, u, s, vh, ws)
    ctx.sync()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        api.svd(ctx, sp, data, u, s, vh, ws)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    x, sv = data.cpu().numpy(), s.cpu().numpy()
    worst, largest = 0.0, (0, 0)
    for (c, r, k, o), (c2, r2, k2, so) in zip(tm.blocks(), sp.blocks()):
        ref = np.linalg.svd(x[o:o + r * k].reshape(k, r).T, compute_uv=False)
        worst = max(worst, float(np.abs(sv[so:so + len(ref)] - ref).max() / max(ref[0], 1e-300)))
        largest = max(largest, (r, k), key=lambda t: t[0] * t[1])
    return {"ms": sorted(times)[len(times) // 2], "blocks": len(sp.blocks()), "largest_block": list(largest),
            "singular_values": nval,
            "max_rel_diff_singular_values_vs_numpy": worst,
            "what": "block SVD of the D = 1024 chain's x' (V (x) P <- V (x) P*), all sectors in one launch"}


def kernels_table(prof, steps):
    return {k: {"launches": c, "ms_per_step": ms / steps} for k, (c, ms) in prof.items()}


def split_roofline(gemm, m, steps):
    """Roofline of the split-precision GEMM launch: executed tensor flops (slice products x the
    block flops routed to the tensor cores) / its event-measured time, against the BF16 peak."""
    work, prof = m["work"], m["prof"]
    kms = prof.get("k_oz_gemm", (0, 0.0))[1]
    if kms <= 0 or work.tensor_flops <= 0:
        return None
    bf = _peaks().get("bf16_tflops")
    if gemm == "ozaki":
        products, peak, src = 21, bf, "measured bf16_tflops (burst)"
    else:  # TF32 dense rate is half of BF16 on this part (nominal 1.1 vs 2.25 PFLOP/s)
        products, peak, src = 3, (bf / 2 if bf else None), "measured bf16_tflops (burst) x 1/2 (nominal TF32:BF16)"
    executed = products * work.tensor_flops * steps / (kms * 1e-3) / 1e12
    return {"kernel": "k_oz_gemm", "bound": "tensor", "achieved": executed, "peak": peak, "unit": "TFLOP/s",
            "frac": executed / peak if peak else None, "traffic": None, "peak_source": src,
            "note": f"achieved = {products} products x tensor-path block flops / k_oz_gemm time"}


def permute_roofline(work, prof, steps):
    kms = prof.get("k_permute", (0, 0.0))[1]
    if kms <= 0:
        return None
    peaks = _peaks()
    pk = peaks.get("hbm_gbs", 6800.0)
    achieved = work.permute_bytes * steps / (kms * 1e-3) / 1e9
    return {"kernel": "k_permute", "bound": "hbm", "achieved": achieved, "peak": pk, "unit": "GB/s",
            "frac": achieved / pk, "traffic": None,
            "peak_source": "measured hbm_gbs" if "hbm_gbs" in peaks else "fallback",
            "note": "algorithmic bytes (every source element read once per use, every output written once) "
                    "/ k_permute time"}


def run_serving(api, local, dist, rank, args, split):
    """The C4 serving loop on its own context (the 150 GB budget covers the server alone):
    calibrate the arrival rate to the offered load, warm up, serve the request stream."""
    from paper_2508_10076_gb300.serve import Server, calibrated_rate, request_stream
    reqs = request_stream(args.serve_requests, seed=1000 + replica_seed(rank))
    serve_ctx = api.Context(local)
    server = Server(serve_ctx, budget_bytes=150 << 30, split_gemm="ozaki" if split else None)
    for r in reqs:
        server.shape(r["sym"], r["D"], r["dtype"])
    rate, mean_s = calibrated_rate(server, reqs, load=args.serve_load)
    server.run(reqs[:200], rate)  # warm-up pass (allocator, first launches)
    _, out, _ = server.run(reqs, rate)
    out["p99_ms"] = max_over_ranks(dist, out["p99_ms"])
    solo = sorted(k for k, sh in server.shapes.items() if sh.solo)
    mem = serve_ctx.memory()
    out.update({"precision": "FP64 (complex128) in packed batches; shapes whose FP64 service alone is >= 1 ms and "
                "faster in Ozaki BF16 (s = 6, <= 1e-10) are served one by one in that mode"
                if split else "FP64 (complex128) in packed batches, every request",
                "split_precision_shapes": len(solo), "shapes": len(server.shapes),
                "plans": "autotuned once per shape before the timed loop",
                "budget_gb": 150, "resident_gb": (mem["library_bytes"] + mem["reserved_bytes"]) / 2**30,
                "budget_counts": "plan tables held by libtk + resident inputs (reserved) + in-flight "
                                 "outputs and workspaces (reserved at admission)",
                "load": args.serve_load, "mean_service_ms_alone": 1e3 * mean_s,
                "mix": "U(1) L.x at D / SU(2) L.x at D/4, D log-uniform 64-4096 "
                       "(25-level grid), half complex128, Poisson arrivals"})
    server.close()
    return out


def run_ours(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(local)
    from paper_2508_10076_gb300 import api, build_library
    build_library()
    ctx = api.Context(local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    timer = Timer(torch, stream, flush, barrier)
    # ---------------- the headline: FP64 on the default workload, clocks sampled
    m = measure(ctx, args.config, args.gemm, args, timer, rank, args.steps, clocks=Clocks(local))
    clk = timer.clk
    # first-call plan construction of the headline chain on a fresh context (structures, fusion
    # trees, recoupling coefficients, work lists, device tables), then the same again on the now
    # warm context (structures and permute plans come from its cache)
    plan_build = None
    if hasattr(m["work"], "plan_build_ms"):
        again = _workload(ctx, args.config, args.gemm, seed=replica_seed(rank))
        plan_build = {"first_ms": round(m["work"].plan_build_ms, 2), "warm_ms": round(again.plan_build_ms, 2),
                      "note": "host time to build every plan of one application, cold context then warm"}
        del again
    work, prof = m["work"], m["prof"]
    flops = work.flops
    total_ms = max_over_ranks(dist, m["total_ms"])
    value = job_throughput(flops, args.steps, world, total_ms)
    # ---------------- end to end: pinned host inputs -> device -> chain -> host result through the
    # C ABI, captured as one graph when the device path is
    ins = _inputs(work)
    host_in = [x.cpu().pin_memory() for x in ins]
    host_out = torch.empty(m["out"].numel(), dtype=m["out"].dtype).pin_memory()
    h2d = sum(x.numel() * x.element_size() for x in host_in)
    d2h = host_out.numel() * host_out.element_size()
    if hasattr(work, "run_host"):
        host_map = dict(zip(("x", "L", "W", "R"), host_in))
        e2e_step = lambda: work.run_host(host_map, host_out)  # noqa: E731
        if m["mode"] == "cuda_graph":
            from paper_2508_10076_gb300.chain import capture_graph
            e2e_graph, _, _ = capture_graph(ctx, e2e_step)
            e2e_step = e2e_graph.replay
    else:
        def e2e_step():
            for hx, dx in zip(host_in, ins):
                api.copy_h2d(ctx, dx, hx.data_ptr(), hx.numel() * hx.element_size(), stream)
            out = work.run()
            api.copy_d2h(ctx, host_out.data_ptr(), out, d2h, stream)
    e2e_ms = max_over_ranks(dist, timer(e2e_step, args.steps, label=f"timed_e2e_{args.config}"))
    torch.cuda.synchronize()
    if not torch.equal(host_out, m["out"].cpu()):
        raise RuntimeError("the end-to-end result differs from the device path's")
    e2e_value = job_throughput(flops, args.steps, world, e2e_ms)
    ctx.sync()
    # ---------------- roofline of the dominant kernel; FP64 peak measured on this GPU now
    probe_clocks = Clocks(local)
    torch.cuda.synchronize()
    probe_clocks.start()
    fp64_peak, fp64_probe_ms = api.probe_fp64_peak(ctx, seconds=1.0)
    probe_clk = probe_clocks.stop()
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else ("none", (0, 0.0))
    kname, (kcount, kms) = dom
    if kname == "k_gemm_f64":
        achieved = flops * args.steps / (kms * 1e-3) / 1e12
        roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak,
                "traffic": K2_TRAFFIC_BYTES.get(args.config) if not args.eager else None,
                "traffic_note": "DRAM bytes per launch (ncu, mean of one application's launches)",
                "peak_source": f"measured in this run: register-only FP64 FMA loop on every SM "
                               f"(tk_probe_fp64_peak, {fp64_probe_ms:.0f} ms)"}
    elif kname == "k_permute":
        roof = permute_roofline(work, prof, args.steps)
    else:
        roof = split_roofline(args.gemm, m, args.steps)
    # ---------------- split-precision variants of the same workload: Ozaki BF16 (s = 6, 21 slice
    # pairs) and 3xTF32 (3 products); error against the FP64 path's output
    variants = {}
    if not args.no_split:
        for gemm in ("ozaki", "tf32x3"):
            v = measure(ctx, args.config, gemm, args, timer, rank, args.steps)
            v_ms = max_over_ranks(dist, v["total_ms"])
            variants[gemm] = {
                "value": job_throughput(flops, args.steps, world, v_ms), "unit": UNIT,
                "ms_per_step": v_ms / args.steps, "roofline": split_roofline(gemm, v, args.steps),
                "autotune": v["tuned"], "tensor_path_flops_per_step": v["work"].tensor_flops,
                "gpu_launches_per_step": v["launches"] / args.steps,
                "rel_frobenius_per_block_vs_fp64_path": rel_err_per_block(
                    _out_blocks(v["work"]), v["out"].cpu().numpy(), m["out"].cpu().numpy()),
                "kernels": kernels_table(v["prof"], args.steps), "out": v["out"]}
            if gemm == "ozaki":
                variants[gemm]["slices"] = 6
        # the same workload at other slice counts (fewer steps): rate against accuracy
        if not args.no_extra:
            sweep = {}
            for sl in (4, 5, 7):
                v = measure(ctx, args.config, "ozaki", args, timer, rank, args.extra_steps, slices=sl)
                v_ms = max_over_ranks(dist, v["total_ms"])
                sweep[str(sl)] = {
                    "value": job_throughput(flops, args.extra_steps, world, v_ms), "unit": UNIT,
                    "ms_per_step": v_ms / args.extra_steps, "slice_pairs": sl * (sl + 1) // 2,
                    "rel_frobenius_per_block_vs_fp64_path": rel_err_per_block(
                        _out_blocks(v["work"]), v["out"].cpu().numpy(), m["out"].cpu().numpy())}
            variants["ozaki"]["slice_sweep"] = sweep
    # ---------------- the other configurations named by the metric (fewer steps)
    extra = {}
    if not args.no_extra:
        for name in EXTRA_CONFIGS:
            if name == args.config:
                continue
            row = {}
            ref_out = None
            for gemm in ("fp64", "ozaki", "tf32x3"):
                e = measure(ctx, name, gemm, args, timer, rank, args.extra_steps)
                e_ms = max_over_ranks(dist, e["total_ms"])
                row[gemm] = {"value": job_throughput(e["work"].flops, args.extra_steps, world, e_ms),
                             "ms_per_step": e_ms / args.extra_steps, "autotune": e["tuned"]}
                if gemm == "fp64":
                    ref_out = e["out"]
                    row["block_flops_per_step"] = e["work"].flops
                    row["permute_roofline"] = permute_roofline(e["work"], e["prof"], args.extra_steps)
                    if hasattr(e["work"], "steps") and name == "c1_u1_heff_d1024":
                        row["block_svd"] = measure_svd(api, ctx, e["work"].steps[-1].out, e["out"], torch)
                else:
                    row[gemm]["rel_frobenius_per_block_vs_fp64_path"] = rel_err_per_block(
                        _out_blocks(e["work"]), e["out"].cpu().numpy(), ref_out.cpu().numpy())
                    row[gemm]["roofline"] = split_roofline(gemm, e, args.extra_steps)
            extra[name] = row
    # ---------------- serving: Poisson stream of mixed requests through the continuous-batching loop,
    # mixed precision (the largest shapes one by one in Ozaki BF16) and FP64 only
    serve = serve_fp64 = None
    if args.serve_requests > 0:
        serve = run_serving(api, local, dist, rank, args, split=True)
        if not args.no_serve_fp64:
            serve_fp64 = run_serving(api, local, dist, rank, args, split=False)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.config, "gemm": args.gemm, "block_flops_per_step": flops,
                   "permute_bytes_per_step": work.permute_bytes,
                   "l2": "flushed (512 MB write) before every timed step",
                   "launch": m["mode"], "autotune": m["tuned"],
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": m["launches"],
        "roofline": roof,
        "roofline_permute": permute_roofline(work, prof, args.steps),
        "fp64_peak_probe": {"tflops": fp64_peak, "ms": fp64_probe_ms, "clocks": probe_clk,
                            "how": "register-only FP64 FMA loop: a 4 x 4 outer product per thread (16 independent "
                                   "chains), 4 CTAs x 256 threads per SM, CUDA events"},
        "kernels": kernels_table(prof, args.steps),
    }
    if plan_build is not None:
        line["plan_build"] = plan_build
    if "ozaki" in variants:
        line["split_precision"] = {k: v for k, v in variants["ozaki"].items() if k != "out"}
    if "tf32x3" in variants:
        line["split_precision_tf32x3"] = {k: v for k, v in variants["tf32x3"].items() if k != "out"}
    if extra:
        line["extra_workloads"] = extra
    if serve is not None:
        line["serve"] = serve
    if serve_fp64 is not None:
        line["serve_fp64"] = serve_fp64
    if world == 1 and not args.no_cpu_baseline:
        n, dt, eff, threads, oracle_out = cpu_baseline(args.config, budget_s=args.cpu_budget)
        line["cpu_baseline"] = {"value": flops * n / dt / 1e9, "unit": UNIT, "cores": round(eff, 1),
                                "threads_available": threads, "kind": "oracle",
                                "sample": f"{n} whole applications of {args.config} by the oracle block tier "
                                          f"({dt:.1f} s); cores = CPU seconds / wall seconds (BLAS threads "
                                          f"in the large sector products, the rest one Python thread)"}
        n1, dt1 = cpu_baseline_single_thread(args.config, budget_s=min(args.cpu_budget, 10.0))
        line["cpu_baseline_single_thread"] = {
            "value": flops * n1 / dt1 / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n1} whole applications of {args.config} by the oracle block tier in a process with "
                      f"one BLAS / OpenMP thread ({dt1:.1f} s)"}
        # every result of the line against the FP64 oracle (seed 0 inputs, rank 0)
        blocks = _out_blocks(work)
        line["rel_frobenius_per_block_vs_oracle"] = {
            "fp64": rel_err_per_block(blocks, m["out"].cpu().numpy(), oracle_out),
            **{g: rel_err_per_block(blocks, v["out"].cpu().numpy(), oracle_out) for g, v in variants.items()}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=DEFAULT_CONFIG)
    ap.add_argument("--gemm", default="fp64", choices=["fp64", "ozaki"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--budget", type=float, default=60.0, help="reference arm: total CPU seconds")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-split", action="store_true", help="skip the split-precision variants")
    ap.add_argument("--no-extra", action="store_true", help="skip the extra workloads")
    ap.add_argument("--extra-steps", type=int, default=10)
    ap.add_argument("--eager", action="store_true", help="launch kernels one by one instead of a CUDA graph")
    ap.add_argument("--serve-requests", type=int, default=10000, help="serving requests (0: skip serving)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the heuristic work lists")
    ap.add_argument("--serve-load", type=float, default=0.7, help="offered load relative to alone service time")
    ap.add_argument("--no-serve-fp64", action="store_true", help="skip the FP64-only serving run")
    ap.add_argument("--cpu-worker", action="store_true", help=argparse.SUPPRESS)  # single-thread baseline process
    args = ap.parse_args()
    if args.cpu_worker:
        n, dt, _, _, _ = cpu_baseline(args.config, budget_s=args.cpu_budget)
        print(json.dumps({"n": n, "dt": dt}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
