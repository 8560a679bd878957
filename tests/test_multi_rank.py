"""The bench's N > 1 path (independent replicas, max-over-ranks time) on CPU: torchrun with two
gloo ranks.  No GPU: the data path has no collective, so the host logic is all there is to test."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, timeout=300):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port())] + args
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-3000:]
    return [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2508_10076_gb300 import build_library
    build_library()


def test_two_gloo_ranks_replica_logic():
    lines = _torchrun([os.path.join("tests", "rank_worker.py")])
    assert len(lines) == 1, lines  # rank 0 alone reports
    d = json.loads(lines[0])
    assert d["world"] == 2
    assert d["slowest"] == 13.0  # max over ranks of 10 + 3 rank
    assert len(set(d["seeds"])) == 2  # independent problems
    assert d["firsts"][0] != d["firsts"][1]
    assert d["flops"][0] == d["flops"][1] > 0  # same shape on every rank
    assert d["value"] == pytest.approx(d["flops"][0] * 4 * 2 / (13.0e-3) / 1e9)


def test_reference_arm_reports_on_rank_zero_only():
    lines = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
                       "--budget", "1", "--config", "c1_u1_heff_d1024"])
    assert len(lines) == 1, lines
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
