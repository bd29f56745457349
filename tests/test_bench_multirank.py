"""The multi-GPU bench path is replicas only: every rank evaluates its own independent
replica, the job's time is the slowest rank's (all-reduce MAX), the value counts every rank's
particles, and ranks other than 0 of the reference arm exit without work.  The host logic runs
here as two gloo ranks on the CPU."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["GB_ROOT"])
import torch, torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, ws = dist.get_rank(), dist.get_world_size()
local_ms = [12.0, 30.0][rank]
tot = bench.max_over_ranks(local_ms, "cpu")
print(json.dumps({"rank": rank, "max": tot, "seed": bench.replica_seed(100, rank),
                  "rate": bench.job_rate(1000, ws, tot, 3)}), flush=True)
dist.destroy_process_group()
"""


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_max_and_rate():
    import json

    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), GB_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    assert [o["max"] for o in outs] == [30.0, 30.0]
    assert outs[0]["seed"] != outs[1]["seed"]
    assert outs[0]["rate"] == pytest.approx(1000 * 2 / (30.0 / 3 / 1e3))


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_single_process_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(7.5, "cpu") == 7.5
    assert bench.job_rate(1 << 20, 1, 2.0, 1) == pytest.approx((1 << 20) / 2e-3)
