"""Benchmark of the symmetric-contraction hot path on GB300 (one JSON line on rank 0).

Default workload: the U(1) two-site effective-Hamiltonian application x' = L.x.W.W.R at
D = 1024 (charges -16..16, n_q ~ exp(-q^2/72)), XXZ MPO, plain FP64 -- four pairwise
contractions, each a fusion-tree permute of both operands, one grouped GEMM over the coupled
sectors and the output permute.  A step is one application of the chain.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config NAME] [--gemm fp64|ozaki]

Under torchrun (N > 1) every rank runs its own replica of the workload (independent problems,
no collective on the data path): value = all ranks' block flops / max-over-ranks time.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "symmetric contraction block-GFLOP/s (FP64 vs split-prec); serve p50/p99 ms"
UNIT = "block-GFLOP/s"
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2
FP64_NOMINAL_GFLOPS = 1250.0  # GB300 FP64, nominal
# DRAM bytes (read + write) per k_gemm_f64 launch of the D = 1024 U(1) heff chain, mean of the four
# launches of one application, from one ncu capture (profiles/k_gemm_f64_u1_heff_d1024_launches.md)
K2_TRAFFIC_BYTES = {"c1_u1_heff_d1024": 7.41e6}


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


def _workload(ctx, name, gemm, dtype="f64", seed=0):
    from paper_2508_10076_gb300 import workloads as wl
    from paper_2508_10076_gb300.chain import HeffChain, LxContraction
    cfg = wl.CONFIGS[name]
    if cfg["kind"] in ("heff", "heff1"):
        return HeffChain(ctx, cfg["sym"], cfg["D"], gemm=gemm, dtype=dtype, seed=seed,
                         sites=2 if cfg["kind"] == "heff" else 1, mpo=cfg.get("mpo"))
    if cfg["kind"] == "lx":
        return LxContraction(ctx, cfg["sym"], cfg["D"], gemm=gemm, dtype=dtype, seed=seed)
    raise SystemExit(f"config {name} is a parity case, not a bench line")


def _inputs_and_output(work):
    from paper_2508_10076_gb300.chain import HeffChain
    if isinstance(work, HeffChain):
        return [work.dev[k] for k in ("x", "L", "W", "R")], (lambda: work.run())
    return [work.dev[k] for k in ("L", "x")], (lambda: work.run())


def cpu_baseline(name, budget_s=15.0):
    """The oracle's block tier on the same workload, repeated for a bounded time on the host."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from harness import oracle_heff, oracle_heff_inputs  # noqa: E402
    from oracle import ops  # noqa: E402
    from paper_2508_10076_gb300 import workloads as wl
    cfg = wl.CONFIGS[name]
    if cfg["kind"] in ("heff", "heff1"):
        sites = 2 if cfg["kind"] == "heff" else 1
        run = lambda: oracle_heff(cfg["sym"], cfg["D"], tier="block", sites=sites, mpo=cfg.get("mpo"))  # noqa: E731
        flops = None
    else:
        st, data = oracle_heff_inputs(cfg["sym"], cfg["D"])
        run = lambda: ops.contract(st["L"], data["L"], *wl.LX_SPEC[:2], st["x"], data["x"],  # noqa: E731
                                   *wl.LX_SPEC[2:], tier="block")
        flops = None
    run()  # warm caches of the oracle
    n, t0 = 0, time.perf_counter()
    while True:
        run()
        n += 1
        if time.perf_counter() - t0 >= budget_s or n >= 200:
            break
    dt = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max((i.get("num_threads", 1) for i in threadpool_info()), default=os.cpu_count())
    except Exception:
        cores = os.cpu_count()
    del flops
    return n, dt, cores


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
    world, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2508_10076_gb300 import workloads as wl
    from paper_2508_10076_gb300.chain import HeffChain, LxContraction  # noqa: F401
    # block flops per step from the host-only planner (no GPU work)
    from paper_2508_10076_gb300 import api, build_library
    build_library()
    hctx = api.Context(-1)
    flops = _host_flops(hctx, args.config)
    per_step = max(1, int(round(args.budget / max(1, args.steps))))
    times = []
    for _ in range(args.warmup):
        cpu_baseline(args.config, budget_s=0.0)
    for _ in range(args.steps):
        n, dt, cores = cpu_baseline(args.config, budget_s=per_step)
        times.append(dt / n)
    ms = 1e3 * statistics.mean(times)
    value = flops / (ms * 1e-3) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.config, "gemm": "fp64 (numpy BLAS)", "tier": "oracle block tier"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"whole {args.config} applications repeated for ~{per_step}s per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _host_flops(hctx, name):
    from paper_2508_10076_gb300 import workloads as wl
    from paper_2508_10076_gb300 import api
    cfg = wl.CONFIGS[name]
    V, P, W = wl.heff_spaces(cfg["sym"], cfg["D"])
    legs = wl.heff_legs(V, P, W) if cfg["kind"] != "heff1" else wl.heff1_legs(V, P, W)

    def tm(k):
        cod, dom = legs[k]
        return hctx.tmap([hctx.space(cfg["sym"], s, d) for s, d in cod], [hctx.space(cfg["sym"], s, d) for s, d in dom])

    if cfg["kind"] == "lx":
        return api.contract_plan(hctx, tm("L"), *wl.LX_SPEC[:2], tm("x"), *wl.LX_SPEC[2:]).flops
    total, cur = 0.0, tm("x")
    specs = wl.HEFF_SPECS if cfg["kind"] != "heff1" else wl.HEFF1_SPECS
    others = ("L", "W", "W", "R") if cfg["kind"] != "heff1" else ("L", "W", "R")
    for i, spec in enumerate(specs):
        if i == 0:
            pl = api.contract_plan(hctx, tm("L"), *spec[:2], cur, *spec[2:])
        else:
            pl = api.contract_plan(hctx, cur, *spec[:2], tm(others[i]), *spec[2:])
        total += pl.flops
        cur = pl.output()
    return total


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
    work = _workload(ctx, args.config, args.gemm, seed=replica_seed(rank))
    tuned = work.autotune() if not args.no_autotune else None  # before any graph capture
    flops = work.flops
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        work.run()
    ctx.sync()
    # one application as a CUDA graph (eager launches if capture is unavailable)
    step_fn, per_step_launches, mode, graph_out = work.run, None, "eager", None
    if not args.eager:
        try:
            graph, graph_out, per_step_launches = work.capture()
            step_fn, mode = graph.replay, "cuda_graph"
            for _ in range(max(3, args.warmup)):
                step_fn()
            torch.cuda.synchronize()
        except Exception as exc:  # keep the eager path; report why
            step_fn, mode = work.run, f"eager (graph capture failed: {exc})"
    # ---------------- timed region: K steps, L2 flushed before each, events around each step
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local)
    barrier()
    clocks.start()
    launches0 = ctx.launches
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        step_fn()
        ends[i].record(stream)
    barrier()
    clk = clocks.stop()
    launches = ctx.launches - launches0 if per_step_launches is None else per_step_launches * args.steps
    ctx.sync()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(dist, total_ms)
    value = job_throughput(flops, args.steps, world, total_ms)
    # ---------------- per-kernel event times: the same loop with libtk's launch profiler on
    ctx.profile(True)
    for i in range(args.steps):
        flush.zero_()
        work.run()
    ctx.sync()
    prof = ctx.profile_read()
    ctx.profile(False)
    # ---------------- end to end: pinned host inputs -> device -> chain -> host result (the chain
    # replayed from its CUDA graph when captured: the graph reads the same input buffers)
    ins, run = _inputs_and_output(work)
    if graph_out is not None:
        run = lambda: (step_fn(), graph_out)[1]  # noqa: E731
    host_in = [x.cpu().pin_memory() for x in ins]
    out_dev = run()
    host_out = torch.empty(out_dev.numel(), dtype=out_dev.dtype).pin_memory()
    h2d = sum(x.numel() * x.element_size() for x in host_in)
    d2h = host_out.numel() * host_out.element_size()
    e2e_step = None
    if hasattr(work, "run_host"):
        # the chain's host-to-host call: W and R copied beside the first contraction
        host_map = dict(zip(("x", "L", "W", "R"), host_in))
        e2e_step = lambda: work.run_host(host_map, host_out)  # noqa: E731
        if graph_out is not None:
            from paper_2508_10076_gb300.chain import capture_graph
            e2e_graph, _, _ = capture_graph(ctx, e2e_step)
            e2e_step = e2e_graph.replay
    e_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_end = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    for i in range(args.steps):
        flush.zero_()
        e_start[i].record(stream)
        if e2e_step is not None:
            e2e_step()
        else:
            for hx, dx in zip(host_in, ins):
                api.copy_h2d(ctx, dx, hx.data_ptr(), hx.numel() * hx.element_size(), stream)
            out_dev = run()
            api.copy_d2h(ctx, host_out.data_ptr(), out_dev, d2h, stream)
        e_end[i].record(stream)
    barrier()
    torch.cuda.synchronize()
    if not torch.equal(host_out, out_dev.cpu() if e2e_step is None else run().cpu()):
        raise RuntimeError("the end-to-end result differs from the device path's")
    e2e_ms = sum(s.elapsed_time(e) for s, e in zip(e_start, e_end))
    e2e_ms = max_over_ranks(dist, e2e_ms)
    e2e_value = job_throughput(flops, args.steps, world, e2e_ms)
    ctx.sync()
    # ---------------- split-precision variants of the same workload on tcgen05: Ozaki BF16 slices
    # (s = 6, 21 slice pairs) and 3xTF32 (3 products, tensor rate half of BF16)
    def split_variant(gemm, ref_out):
        oz = _workload(ctx, args.config, gemm, seed=replica_seed(rank))
        oz_tuned = oz.autotune() if not args.no_autotune else None
        for _ in range(max(3, args.warmup)):
            oz.run()
        oz_fn = oz.run
        if mode == "cuda_graph":
            oz_graph, _, _ = oz.capture()
            oz_fn = oz_graph.replay
            for _ in range(max(3, args.warmup)):
                oz_fn()
        o_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        o_end = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        barrier()
        for i in range(args.steps):
            flush.zero_()
            o_start[i].record(stream)
            oz_fn()
            o_end[i].record(stream)
        barrier()
        oz_ms = sum(s.elapsed_time(e) for s, e in zip(o_start, o_end))
        oz_ms = max_over_ranks(dist, oz_ms)
        oz_out = oz.run()
        ctx.profile(True)
        for i in range(args.steps):
            flush.zero_()
            oz.run()
        ctx.sync()
        oz_prof = ctx.profile_read()
        ctx.profile(False)
        out_blocks = (oz.steps[-1].out if hasattr(oz, "steps") else oz.step.out).blocks()
        worst = 0.0
        refn = float(torch.linalg.norm(ref_out))
        for _, r_, k_, o_ in out_blocks:
            d = float(torch.linalg.norm(oz_out[o_:o_ + r_ * k_] - ref_out[o_:o_ + r_ * k_]))
            n_ = float(torch.linalg.norm(ref_out[o_:o_ + r_ * k_]))
            worst = max(worst, d / (n_ if n_ > 1e-13 * refn else refn))
        oz_kms = oz_prof.get("k_oz_gemm", (0, 0.0))[1]
        if gemm == "ozaki":
            products, peak, peak_key = 21, _peaks().get("bf16_tflops"), "measured bf16_tflops (burst)"
        else:  # TF32 dense rate is half of BF16 on this part (nominal 1.1 vs 2.25 PFLOP/s)
            bf = _peaks().get("bf16_tflops")
            products, peak, peak_key = 3, (bf / 2 if bf else None), "measured bf16_tflops (burst) x 1/2 (nominal TF32:BF16)"
        roof = None
        if oz_kms > 0 and oz.tensor_flops > 0:
            executed = products * oz.tensor_flops * args.steps / (oz_kms * 1e-3) / 1e12
            roof = {"kernel": "k_oz_gemm", "bound": "tensor", "achieved": executed, "peak": peak,
                    "unit": "TFLOP/s", "frac": executed / peak if peak else None, "traffic": None,
                    "peak_source": peak_key,
                    "note": f"achieved = {products} products x tensor-path block flops / k_oz_gemm time"}
        return {"value": job_throughput(flops, args.steps, world, oz_ms), "unit": UNIT,
                "ms_per_step": oz_ms / args.steps, "roofline": roof, "autotune": oz_tuned,
                "tensor_path_flops_per_step": oz.tensor_flops,
                "rel_frobenius_per_block_vs_fp64_path": worst,
                "kernels": {k: {"launches": c, "ms_per_step": ms / args.steps} for k, (c, ms) in oz_prof.items()}}

    split = tf32 = None
    if not args.no_split:
        ref_out = run().clone()
        split = split_variant("ozaki", ref_out)
        split["slices"] = 6
        tf32 = split_variant("tf32x3", ref_out)
    # ---------------- serving: Poisson stream of mixed requests through the continuous-batching loop
    serve = None
    if args.serve_requests > 0:
        from paper_2508_10076_gb300.serve import Server, calibrated_rate, request_stream
        reqs = request_stream(args.serve_requests, seed=1000 + replica_seed(rank))
        server = Server(ctx, budget_bytes=150 << 30, split_gemm=None if args.serve_fp64 else "ozaki")
        for r in reqs:
            server.shape(r["sym"], r["D"], r["dtype"])
        rate, mean_s = calibrated_rate(server, reqs, load=args.serve_load)
        server.run(reqs[:200], rate)  # warm-up pass (allocator, first launches)
        _, serve, _ = server.run(reqs, rate)
        serve["p99_ms"] = max_over_ranks(dist, serve["p99_ms"])
        solo = sorted(k for k, sh in server.shapes.items() if sh.solo)
        serve.update({"precision": "FP64 (complex128) in packed batches; shapes whose FP64 service alone is >= 1 ms and "
                      "faster in Ozaki BF16 (s = 6, <= 1e-10) are served one by one in that mode"
                      if not args.serve_fp64 else "FP64 (complex128) in packed batches",
                      "split_precision_shapes": len(solo), "shapes": len(server.shapes)})
        serve.update({"load": args.serve_load, "mean_service_ms_alone": 1e3 * mean_s,
                      "budget_gb": 150, "mix": "U(1) L.x at D / SU(2) L.x at D/4, D log-uniform 64-4096 "
                      "(25-level grid), half complex128, Poisson arrivals"})
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    # ---------------- roofline of the dominant kernel
    peaks = _peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else ("none", (0, 0.0))
    kname, (kcount, kms) = dom
    permute_bytes = work.permute_bytes
    if kname == "k_gemm_f64":
        achieved = flops * args.steps / (kms * 1e-3) / 1e12
        roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_GFLOPS / 1e3,
                "unit": "TFLOP/s", "frac": achieved / (FP64_NOMINAL_GFLOPS / 1e3),
                "traffic": K2_TRAFFIC_BYTES.get(args.config) if not args.eager else None,
                "traffic_note": "DRAM bytes per launch (ncu); operands read once, outputs written back after the launch",
                "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s); no FP64 figure in MEASURED_PEAKS.json"}
    elif kname == "k_permute":
        achieved = permute_bytes * args.steps / (kms * 1e-3) / 1e9
        pk = peaks.get("hbm_gbs", 6800.0)
        roof = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": pk, "unit": "GB/s",
                "frac": achieved / pk, "traffic": None, "peak_source": "measured hbm_gbs" if "hbm_gbs" in peaks else "fallback"}
    else:
        roof = {"kernel": kname, "bound": "tensor", "achieved": None, "peak": peaks.get("bf16_tflops"),
                "unit": "TFLOP/s", "frac": None, "traffic": None}
    kernels = {k: {"launches": c, "ms_per_step": ms / args.steps} for k, (c, ms) in prof.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.config, "gemm": args.gemm, "block_flops_per_step": flops,
                   "permute_bytes_per_step": permute_bytes, "l2": "flushed (512 MB write) before every timed step",
                   "launch": mode, "autotune": tuned,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "kernels": kernels,
    }
    if split is not None:
        line["split_precision"] = split
    if tf32 is not None:
        line["split_precision_tf32x3"] = tf32
    if serve is not None:
        line["serve"] = serve
    if world == 1 and not args.no_cpu_baseline:
        n, dt, cores = cpu_baseline(args.config, budget_s=args.cpu_budget)
        line["cpu_baseline"] = {"value": flops * n / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{n} whole applications of {args.config} by the oracle block tier "
                                          f"({dt:.1f} s)"}
        n1, dt1 = cpu_baseline_single_thread(args.config, budget_s=min(args.cpu_budget, 10.0))
        line["cpu_baseline_single_thread"] = {
            "value": flops * n1 / dt1 / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n1} whole applications of {args.config} by the oracle block tier in a process with "
                      f"one BLAS / OpenMP thread ({dt1:.1f} s)"}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c1_u1_heff_d1024")
    ap.add_argument("--gemm", default="fp64", choices=["fp64", "ozaki"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--budget", type=float, default=60.0, help="reference arm: total CPU seconds")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-split", action="store_true", help="skip the split-precision variant")
    ap.add_argument("--eager", action="store_true", help="launch kernels one by one instead of a CUDA graph")
    ap.add_argument("--serve-requests", type=int, default=10000, help="serving requests (0: skip serving)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the heuristic work lists")
    ap.add_argument("--serve-load", type=float, default=0.7, help="offered load relative to alone service time")
    ap.add_argument("--serve-fp64", action="store_true", help="serve every request in FP64 (no split-precision solo path)")
    ap.add_argument("--cpu-worker", action="store_true", help=argparse.SUPPRESS)  # single-thread baseline process
    args = ap.parse_args()
    if args.cpu_worker:
        n, dt, _ = cpu_baseline(args.config, budget_s=args.cpu_budget)
        print(json.dumps({"n": n, "dt": dt}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
