"""The multi-GPU shards' arithmetic on one GPU, through the C ABI.

Bands of rows (paper_1401_0427_gb300/decomposition.py), stepped one after the other in one
process with the ghost rows refreshed by direct copies (lbm_sw_get_rows / lbm_sw_set_rows),
must give the undivided grid's state bit for bit: the same kernels (the fused K = 6 kernel
on bands large enough for it) on the same values.  Their row-window diagnostics
(lbm_sw_diagnostics_rows) add up to the whole grid's.  A batch over a subset of instances
(the shard of the instance list) gives the full batch's instances bit for bit."""

import numpy as np
import pytest

from paper_1401_0427_gb300 import decomposition as dc
from paper_1401_0427_gb300 import inputs, lbm_sw

from gpu_helpers import torch_stream

pytestmark = pytest.mark.gpu

P, W, O, I = lbm_sw.PERIODIC, lbm_sw.WALL, lbm_sw.OUTFLOW, lbm_sw.INFLOW
INFLOW = [(1.1, 0.1, 0.0), (1.0, 0.0, 0.0), (1.05, 0.0, 0.08), (1.0, 0.0, 0.0)]


def _split_run(nx, ny, world, halo, steps, bc, precision, W0):
    bands = [dc.Band(nx, ny, r, world, halo=halo, bc=bc, precision=precision, inflow=INFLOW, stream=torch_stream())
             for r in range(world)]
    for b in bands:
        b.set_state(*W0)
    strips = dc.LocalStrips(bands)
    strips.step(steps)
    h = np.concatenate([b.moments()[0] for b in bands])
    hu = np.concatenate([b.moments()[1] for b in bands])
    diags = [b.local_diagnostics() for b in bands]
    info = [b.sim.info() for b in bands]
    for b in bands:
        b.sim.close()
    return h, hu, diags, info


def _whole_run(nx, ny, steps, bc, precision, W0):
    with lbm_sw.Simulation(nx, ny, precision=precision, bc=bc, inflow=INFLOW, stream=torch_stream()) as sim:
        sim.set_state(*W0)
        sim.step(steps)
        h, hu, _ = sim.moments()
        return h, hu, sim.diagnostics()


@pytest.mark.parametrize("nx,ny,world,halo,steps,bc,precision", [
    (2048, 2048, 4, 6, 40, (P, P, P, P), lbm_sw.FP32),   # bands of 512 + 12 rows: the fused kernel
    (2048, 2048, 3, 6, 23, (P, P, W, W), lbm_sw.FP32),
    (1024, 768, 3, 4, 21, (I, O, W, O), lbm_sw.FP64),
    (300, 97, 5, 3, 14, (P, P, P, P), lbm_sw.FP64),
    (301, 96, 2, 6, 31, (W, W, I, W), lbm_sw.FP32),
])
def test_bands_equal_the_undivided_grid(nx, ny, world, halo, steps, bc, precision):
    W0 = inputs.circular_dam_break_2d(max(nx, ny), seed=inputs.stream_seed(3, nx))
    W0 = [np.ascontiguousarray(w[:ny, :nx]) for w in W0]
    h, hu, diags, info = _split_run(nx, ny, world, halo, steps, bc, precision, W0)
    wh, whu, wd = _whole_run(nx, ny, steps, bc, precision, W0)
    assert np.array_equal(h, wh) and np.array_equal(hu, whu)
    if nx * ny >= 2048 * 2048 and precision == lbm_sw.FP32:
        assert all(i.steps_per_launch == 6 for i in info)
    total = [sum(d[k] for d in diags) for k in range(3)]
    for k in range(3):
        assert abs(total[k] - wd[k]) <= 1e-12 * abs(wd[0])
    assert min(d[3] for d in diags) == wd[3]


def test_rows_round_trip_and_window_diagnostics():
    import torch

    nx, ny = 130, 40
    W0 = [x.reshape(ny, nx) for x in inputs.random_states(nx * ny, seed=31, h=(0.8, 1.4), speed=0.25)]
    with lbm_sw.Simulation(nx, ny, stream=torch_stream()) as sim:
        sim.set_state(*W0)
        sim.step(3)
        F = sim.populations()
        rows = torch.empty((13, 7, nx), dtype=torch.float32, device="cuda")
        sim.get_rows_into(10, 7, rows)
        assert np.array_equal(rows.cpu().numpy(), F[:, 10:17])
        host = np.empty((13, 7, nx), np.float32)
        sim.get_rows_into(10, 7, host)
        assert np.array_equal(host, F[:, 10:17])
        sim.set_rows(0, 7, rows)  # rows 10..16 copied over rows 0..6
        G = sim.populations()
        assert np.array_equal(G[:, :7], F[:, 10:17]) and np.array_equal(G[:, 7:], F[:, 7:])
        d = sim.diagnostics_rows(10, 7)
        # depth of each cell in the storage precision, summed in mirror pairs as the kernels do
        h = (G[0] + ((G[1] + G[3]) + (G[2] + G[4])))[10:17].astype(np.float64)
        assert abs(d[0] - h.sum()) <= 1e-12 * h.sum() and d[3] == h.min()
        with pytest.raises(lbm_sw.LbmSwError):
            sim.get_rows_into(35, 7, rows)
        with pytest.raises(lbm_sw.LbmSwError):
            sim.diagnostics_rows(-1, 3)


def test_instance_shards_equal_the_full_batch():
    table = inputs.batched_instances(256)[:24]
    sizes = [(n, n) for n, _, _ in table]
    states = [inputs.circular_dam_break_2d(n, seed=None, h_in=hin, radius=r) for n, hin, r in table]
    with lbm_sw.Batch(sizes, stream=torch_stream()) as b:
        for i, W0 in enumerate(states):
            b.set_state(i, *W0)
        b.step(30)
        want = [b.populations(i) for i in range(len(sizes))]
    for part in dc.partition_instances([nx * ny for nx, ny in sizes], 3):
        with lbm_sw.Batch([sizes[i] for i in part], stream=torch_stream()) as b:
            for k, i in enumerate(part):
                b.set_state(k, *states[i])
            b.step(30)
            for k, i in enumerate(part):
                assert np.array_equal(b.populations(k), want[i]), i
