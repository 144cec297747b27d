"""The multi-rank path of bench.py on CPU: two gloo ranks (one process each, as under
torchrun) check the barrier, the max and sum reductions and the whole-job throughput of
replicas (the units of every rank over the slowest rank's time); the reference arm prints
on rank 0 only."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
world, rank, local = bench.dist_setup()
bench.barrier(world)
out = {
    "world": world, "rank": rank,
    "max": bench.max_over_ranks(world, float(rank + 1)),
    "sum": bench.sum_over_ranks(world, 10.0 * (rank + 1)),
    "job": bench.job_throughput(world, 1e6 * (rank + 1), 2.0 + rank),
}
bench.barrier(world)
dist.destroy_process_group()
print(json.dumps(out))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(code, world, extra_env=None):
    port = _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code] if code else extra_env["ARGS"].split(),
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            p.kill()
            raise
        assert p.returncode == 0, e[-2000:]
        outs.append(o)
    return outs


def test_two_gloo_ranks_reduce_and_compute_the_job_throughput():
    outs = [json.loads(o.strip().splitlines()[-1]) for o in _launch(RANK_SCRIPT, 2)]
    for r, o in enumerate(outs):
        assert o["world"] == 2 and o["rank"] == r
        assert o["max"] == 2.0 and o["sum"] == 30.0
        value, slowest = o["job"]
        assert slowest == 3.0
        assert value == pytest.approx((1e6 + 2e6) / 3e-3 / 1e6)


def test_reference_arm_prints_on_rank_zero_only():
    outs = _launch(None, 2, {"ARGS": f"{sys.executable} bench.py --impl reference --steps 1 --warmup 3"})
    lines = [[l for l in o.splitlines() if l.startswith("{")] for o in outs]
    assert len(lines[0]) == 1 and len(lines[1]) == 0
    line = json.loads(lines[0][0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 1
