"""The N > 1 launch path on the CPU (gloo, world size 2).

With N GPUs the bench runs N replicas, one rank each, with no data-path
collective. The only cross-rank steps are the timing reductions: the slowest
rank's time is taken (max over ranks), and whole-job throughput counts every
rank's replica. These tests run those steps on gloo ranks. They also launch
the reference arm under torch.distributed.run with two processes: rank 0
alone prints one JSON line, and the other rank exits 0 without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank           # rank 1 is the slow one
        slowest = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        dist.barrier()
        out[rank] = slowest
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_takes_the_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert dict(out) == {0: 15.0, 1: 15.0}


def test_job_throughput_counts_every_replica():
    # two replicas of 2,197,000 DoF, 5 steps in 0.25 s
    assert bench.job_throughput(2, 2_197_000, 5, 0.25) == pytest.approx(2 * 2_197_000 * 5 / 0.25)


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
