"""The multi-GPU shards on the host: a grid split into bands of rows over gloo ranks (one
process each, as under torchrun), and the batch's instances split over ranks.

Each band's stepper is the FP64 oracle (tests/decomp_helpers.py), so the halo exchange, the
ghost-row layout and the diagnostics' all-reduce run exactly as on GPUs, and the bands'
own rows must equal the undivided oracle run bit for bit: the scheme moves every population
one cell per step (section 3, Eq. 3-stencil-d2q5), so at most H steps between exchanges
leave the band's rows untouched by its ghost rows' open sides."""

import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1401_0427_gb300 import decomposition as dc
from paper_1401_0427_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P, W, O, I = 0, 1, 2, 3
INFLOW = [(1.1, 0.1, 0.0), (1.0, 0.0, 0.0), (1.05, 0.0, 0.08), (1.0, 0.0, 0.0)]

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"]); sys.path.insert(0, os.path.join(os.environ["ROOT"], "tests"))
import numpy as np
import torch.distributed as dist
from paper_1401_0427_gb300 import decomposition as dc
from decomp_helpers import OracleStepper
case = json.loads(os.environ["CASE"])
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
nx, ny, halo, bc = case["nx"], case["ny"], case["halo"], tuple(case["bc"])
L = dc.layout(ny, world, rank, halo, bc)
band = dc.Band(nx, ny, rank, world, halo=halo, bc=bc,
               stepper=OracleStepper(nx, L.local_ny, bc=L.bc, inflow=case["inflow"]))
strips = dc.DistributedStrips(band, device="cpu")
W0 = [np.load(os.path.join(case["dir"], f"w{k}.npy")) for k in range(3)]
band.set_state(*W0)
strips.step(case["steps"])
h, hu, hv = band.moments()
np.save(os.path.join(case["dir"], f"band{rank}.npy"), np.stack([h, hu, hv]))
diag = strips.diagnostics()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "y0": L.y0, "y1": L.y1, "diag": diag, "oracle_steps": band.sim.steps}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(case, world):
    port = _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="", CASE=json.dumps(case),
                   OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=180)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, e[-3000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    return outs


CASES = [
    # world, nx, ny, halo, steps, bc
    (2, 40, 30, 3, 11, (P, P, P, P)),
    (3, 33, 29, 4, 13, (P, P, W, W)),
    (2, 24, 20, 2, 9, (I, O, W, O)),
    (4, 16, 24, 3, 10, (W, W, P, P)),
    (3, 20, 31, 5, 17, (O, I, I, W)),
]


@pytest.mark.parametrize("world,nx,ny,halo,steps,bc", CASES)
def test_bands_over_gloo_ranks_equal_the_undivided_grid(tmp_path, world, nx, ny, halo, steps, bc):
    W0 = [x.reshape(ny, nx) for x in inputs.random_states(nx * ny, seed=900 + nx + ny, h=(0.8, 1.4), speed=0.25)]
    for k, w in enumerate(W0):
        np.save(tmp_path / f"w{k}.npy", w)
    case = {"nx": nx, "ny": ny, "halo": halo, "bc": list(bc), "steps": steps, "inflow": INFLOW,
            "dir": str(tmp_path)}
    outs = _run_ranks(case, world)
    p = oracle.params(nx, ny, a=0.05, bc=bc, inflow=INFLOW)
    want = np.stack(oracle.moments_2d(oracle.run_2d(oracle.equilibrium_2d(*W0, p), steps, p), p))
    got = np.concatenate([np.load(tmp_path / f"band{o['rank']}.npy") for o in sorted(outs, key=lambda o: o["y0"])],
                         axis=1)
    assert got.shape == want.shape
    assert np.array_equal(got, want)
    assert [o["y0"] for o in outs] == [dc.band_rows(ny, world, r)[0] for r in range(world)]
    for o in outs:
        s0, s1, s2, mn, bad = o["diag"]
        assert bad == 0 and mn == want[0].min()
        for v, w in zip((s0, s1, s2), want):
            assert abs(v - w.sum()) <= 1e-13 * np.abs(want[0]).sum()
        assert o["oracle_steps"] == steps


def test_band_rows_cover_the_grid_evenly():
    for ny in (1, 7, 30, 4096, 4097):
        for world in range(1, 9):
            rows = [dc.band_rows(ny, world, r) for r in range(world)]
            assert rows[0][0] == 0 and rows[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
            sizes = [y1 - y0 for y0, y1 in rows]
            assert max(sizes) - min(sizes) <= 1


def test_layout_of_the_bands():
    L = dc.layout(4096, 8, 0, 6, (P, P, P, P))
    assert (L.lo, L.hi, L.down, L.up, L.local_ny) == (6, 6, 7, 1, 512 + 12) and L.bc == (P, P, O, O)
    L = dc.layout(4096, 8, 0, 6, (P, P, W, I))
    assert (L.lo, L.hi, L.down, L.up) == (0, 6, None, 1) and L.bc == (P, P, W, O)
    L = dc.layout(4096, 8, 7, 6, (P, P, W, I))
    assert (L.lo, L.hi, L.down, L.up) == (6, 0, 6, None) and L.bc == (P, P, O, I)
    L = dc.layout(100, 1, 0, 6, (P, P, P, P))
    assert (L.lo, L.hi, L.local_ny, L.bc) == (0, 0, 100, (P, P, P, P))
    with pytest.raises(ValueError, match="fewer than"):
        dc.layout(20, 5, 0, 6, (P, P, P, P))


def test_partition_instances_balances_independent_grids():
    table = inputs.batched_instances(256)
    cells = [n * n for n, _, _ in table]
    for world in (1, 2, 3, 4, 8):
        parts = dc.partition_instances(cells, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(cells)))
        loads = [sum(cells[i] for i in p) for p in parts]
        assert max(loads) <= sum(cells) / world + max(cells)
        assert dc.partition_instances(cells, world) == parts  # deterministic
    assert dc.partition_instances([5, 3, 9], 2) == [[2], [0, 1]]  # 9 first to rank 0, then 5 and 3 to rank 1
