"""The benchmark's multi-rank bookkeeping on CPU with two gloo ranks: a
job's time is its slowest rank's, throughput counts every rank's units, and
the reference arm runs on rank 0 only (replicas: no data-path collective)."""
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


CHILD = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"])
dist.init_process_group("gloo")
dt = bench._max_over_ranks(torch, dist, 1.0 + rank, "cpu")   # ranks took 1 s and 2 s
rate = bench._job_rate(1000, int(os.environ["WORLD_SIZE"]), dt)
print(f"rank {{rank}} dt {{dt}} rate {{rate}}", flush=True)
dist.barrier()
dist.destroy_process_group()
"""


def _run_two(code):
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_two_gloo_ranks_job_time_is_the_slowest():
    outs = _run_two(CHILD.format(root=ROOT))
    for o in outs:
        assert "dt 2.0 rate 1000.0" in o, o


def test_reference_arm_only_on_rank_zero():
    """Under torchrun every rank but 0 leaves at once, printing nothing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
