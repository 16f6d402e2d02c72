"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): replicas, max over ranks,
and the reference arm running on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
local_ms = 100.0 * (rank + 1)                  # rank 1 is the slowest
m = bench.max_over_ranks_ms(local_ms, dist)
v = bench.whole_job_value(world, 4, 0.25, m)
print(json.dumps({{"rank": rank, "max_ms": m, "value": v}}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _launch(code, world=2):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_max_over_ranks_and_whole_job_value():
    outs = _launch(WORKER.format(root=ROOT))
    recs = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for r in recs:
        assert r["max_ms"] == 200.0
        assert abs(r["value"] - 2 * 4 * 0.25 / 0.2) < 1e-12


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
