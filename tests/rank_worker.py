"""One rank of the bench's multi-rank host logic, run under torchrun with the gloo backend on CPU.

Checks: the max-over-ranks reduction of step times, distinct per-rank inputs, identical block
flops per step on every rank (so the whole-job throughput is flops x steps x world / slowest
time), and that only rank 0 reports.  Prints one JSON line on rank 0.
"""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    slowest = bench.max_over_ranks(dist, 10.0 + 3.0 * rank)
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.replica_seed(rank))
    flops = bench.oracle_block_flops("c1_u1_heff_d1024")
    all_flops = [None] * world
    dist.all_gather_object(all_flops, flops)
    from paper_2508_10076_gb300.chain import HeffChain  # noqa: F401  (import only: no device here)
    from paper_2508_10076_gb300 import workloads as wl
    first = wl.normal(16 * bench.replica_seed(rank), 8).tolist()
    firsts = [None] * world
    dist.all_gather_object(firsts, first)
    if rank == 0:
        print(json.dumps({"world": world, "slowest": slowest, "seeds": seeds, "flops": all_flops,
                          "firsts": firsts,
                          "value": bench.job_throughput(flops, 4, world, slowest)}), flush=True)
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
