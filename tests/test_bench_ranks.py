"""Host logic of bench.py's multi-process runs (N independent replicas, one per GPU; the step
does not shard), on the CPU with the gloo backend and two ranks: the slowest rank's timings
reach every rank, the job throughput counts every replica, and under torchrun the reference
arm runs on rank 0 only."""
import argparse
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"]); world = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
got = bench.max_over_ranks([10.0 + 5.0 * rank, 3.0 - rank], world, "cpu")
print(json.dumps({"rank": rank, "got": got, "value": bench.job_throughput(world, got[0] * 1e-3)}))
dist.destroy_process_group()
"""


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_slowest_rank_timing_reaches_every_rank():
    world, port = 2, free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), REPO_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        # rank 1 is the slower one in the first entry, rank 0 in the second
        assert o["got"] == [15.0, 3.0]
        assert o["value"] == pytest.approx(2 / 15e-3)


def test_job_throughput_counts_replicas():
    import bench
    assert bench.job_throughput(1, 0.2) == pytest.approx(5.0)
    assert bench.job_throughput(8, 0.2) == pytest.approx(40.0)
    assert bench.max_over_ranks([1.5, 2.5], 1, "cpu") == [1.5, 2.5]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(argparse.Namespace(steps=1, warmup=0, gpus=2), dict(bench.WORKLOAD))
    assert capsys.readouterr().out == ""
