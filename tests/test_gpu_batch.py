"""Batched instances (one persistent launch per step over a tile list) against single
handles and the oracle.

Every instance of a batch runs the device code of the single-grid kernel, so after n
steps its populations must equal those of its own handle bit for bit, whatever tile
shape and schedule the batch uses; a subset is also compared with the oracle.  The
benchmark's instance table (256 dam-breaks, sides 64..1024) is checked at full size
for a few instances.
"""

import numpy as np
import pytest

import oracle
from paper_1401_0427_gb300 import inputs, lbm_sw

from gpu_helpers import FP32_L1_TOL, FP64_TOL, rel_l1, rel_max, torch_stream

pytestmark = pytest.mark.gpu

P, W, O, I = lbm_sw.PERIODIC, lbm_sw.WALL, lbm_sw.OUTFLOW, lbm_sw.INFLOW
SIZES = [(1, 1), (3, 2), (7, 5), (64, 64), (130, 9), (257, 33), (100, 200), (513, 3)]
INFLOW = [(1.3, 0.2, -0.1), (0.9, -0.15, 0.05), (1.1, 0.05, 0.12), (1.2, -0.08, -0.2)]


def _states(sizes, seed):
    out = []
    for k, (nx, ny) in enumerate(sizes):
        h, hu, hv = inputs.random_states(nx * ny, seed=seed + k, h=(0.7, 1.6), speed=0.3)
        out.append(tuple(x.reshape(ny, nx) for x in (h, hu, hv)))
    return out


def _single(nx, ny, W0, steps, precision, bc):
    with lbm_sw.Simulation(nx, ny, precision=precision, bc=bc, inflow=INFLOW, stream=torch_stream()) as sim:
        sim.set_state(*W0)
        sim.step(steps)
        return sim.populations()


@pytest.mark.parametrize("precision", [lbm_sw.FP32, lbm_sw.FP64])
@pytest.mark.parametrize("bc", [(P, P, P, P), (W, O, I, W)], ids=["PPPP", "WOIW"])
@pytest.mark.parametrize("tile_rows,ctas", [(1, 2), (2, 16), (4, 0), (8, 8)])
def test_batch_equals_single_handles_bitwise(precision, bc, tile_rows, ctas):
    steps = 9
    states = _states(SIZES, seed=700)
    with lbm_sw.Batch(SIZES, precision=precision, bc=bc, inflow=INFLOW, stream=torch_stream(), tile_rows=tile_rows,
                      ctas_per_sm=ctas, graph_chunk=4) as batch:
        for i, W0 in enumerate(states):
            batch.set_state(i, *W0)
        batch.step(steps)  # two graph replays + one single launch
        for i, ((nx, ny), W0) in enumerate(zip(SIZES, states)):
            assert np.array_equal(batch.populations(i), _single(nx, ny, W0, steps, precision, bc)), (i, nx, ny)


def test_batch_fp64_matches_oracle():
    steps = 12
    bc = (W, O, I, W)
    sizes = SIZES[:6]
    states = _states(sizes, seed=900)
    with lbm_sw.Batch(sizes, precision=lbm_sw.FP64, bc=bc, inflow=INFLOW, stream=torch_stream()) as batch:
        for i, W0 in enumerate(states):
            batch.set_state(i, *W0)
        batch.step(steps)
        for i, ((nx, ny), W0) in enumerate(zip(sizes, states)):
            p = oracle.params(nx, ny, a=0.05, bc=bc, inflow=INFLOW)
            want = oracle.moments_2d(oracle.run_2d(oracle.equilibrium_2d(*W0, p), steps, p), p)
            got = batch.moments(i)
            assert rel_max(got[0], want[0]) <= FP64_TOL
            assert max(np.abs(got[1] - want[1]).max(), np.abs(got[2] - want[2]).max()) <= FP64_TOL * np.abs(want[0]).max()


def test_autotune_keeps_the_state_and_picks_a_candidate():
    states = _states(SIZES, seed=1100)
    with lbm_sw.Batch(SIZES, stream=torch_stream()) as batch:
        for i, W0 in enumerate(states):
            batch.set_state(i, *W0)
        batch.step(3)
        before = [batch.populations(i) for i in range(len(SIZES))]
        t = batch.autotune(3)
        # 16 one-step shapes and schedules, then temporal blocking at K = 4, 6, 8
        assert t.candidates == 16 + 3 and t.tile_rows in (1, 2, 4, 8) and t.ctas_per_sm in (0, 2, 4, 8)
        assert t.temporal_steps in (1, 4, 6, 8)
        assert t.ms_per_step > 0 and t.cells == sum(nx * ny for nx, ny in SIZES)
        for i in range(len(SIZES)):
            assert np.array_equal(batch.populations(i), before[i])
        batch.step(5)
        for i, ((nx, ny), W0) in enumerate(zip(SIZES, states)):
            assert np.array_equal(batch.populations(i), _single(nx, ny, W0, 8, lbm_sw.FP32, (P,) * 4))


def test_batch_errors():
    with lbm_sw.Batch([(8, 8), (16, 4)], stream=torch_stream()) as batch:
        batch.set_state(0, np.ones((8, 8)), np.zeros((8, 8)), np.zeros((8, 8)))
        with pytest.raises(lbm_sw.LbmSwError) as ei:
            batch.step(1)
        assert ei.value.status == lbm_sw.E_STATE and "1 of 2" in str(ei.value)
        with pytest.raises(lbm_sw.LbmSwError) as ei:
            batch.set_state(2, np.ones((4, 16)), np.zeros((4, 16)))
        assert ei.value.status == lbm_sw.E_ARG


def test_benchmark_instance_table_full_size():
    """The 256 dam-breaks (sides 64..1024, depth in [1.5, 4], radius in [0.1, 0.3]) for 500
    steps in FP32: a few instances against their own handles (bitwise) and the smallest
    against the FP64 oracle (relative L1 of h)."""
    table = inputs.batched_instances(256)
    sizes = [(n, n) for n, _, _ in table]
    states = [inputs.circular_dam_break_2d(n, seed=None, h_in=hin, radius=r) for n, hin, r in table]
    steps = 500
    with lbm_sw.Batch(sizes, stream=torch_stream()) as batch:
        for i, W0 in enumerate(states):
            batch.set_state(i, *W0)
        batch.autotune(3)
        batch.step(steps)
        order = np.argsort([n for n, _, _ in table])
        picks = [int(order[0]), int(order[-1]), int(order[len(order) // 2]), 17]
        for i in picks:
            n = sizes[i][0]
            assert np.array_equal(batch.populations(i), _single(n, n, states[i], steps, lbm_sw.FP32, (P,) * 4)), i
        i = int(order[0])
        n = sizes[i][0]
        p = oracle.params(n, n, a=0.05)
        want = oracle.moments_2d(oracle.run_2d(oracle.equilibrium_2d(*states[i], p), steps, p), p)
        assert rel_l1(batch.moments(i)[0], want[0]) <= FP32_L1_TOL
        for i in range(0, 256, 37):
            d = batch.diagnostics(i)
            assert d[4] == lbm_sw.OK


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6, 7, 8])
def test_batch_temporal_equals_one_step_per_launch(k):
    """Temporal blocking over the batch's work list (instance, strip, row segment) against one
    tile-list launch per step: the same arithmetic, so the same bits, for odd and even sizes,
    instances narrower than a strip and wider than several."""
    sizes = [(1, 1), (3, 2), (7, 5), (64, 64), (130, 9), (257, 33), (100, 200), (513, 3), (400, 37), (181, 181)]
    states = _states(sizes, seed=1300 + k)
    out = []
    for temporal in (1, k):
        with lbm_sw.Batch(sizes, stream=torch_stream(), temporal_steps=temporal) as batch:
            for i, W0 in enumerate(states):
                batch.set_state(i, *W0)
            batch.step(2 * k + 3)
            assert batch.tuning().temporal_steps == temporal
            out.append([batch.populations(i) for i in range(len(sizes))])
    for i in range(len(sizes)):
        assert np.array_equal(out[0][i], out[1][i]), (k, sizes[i])


def test_batch_temporal_on_the_benchmark_table_and_autotune():
    table = inputs.batched_instances(256)[:48]
    sizes = [(n, n) for n, _, _ in table]
    states = [inputs.circular_dam_break_2d(n, seed=None, h_in=hin, radius=r) for n, hin, r in table]
    out = []
    for temporal in (1, 0):
        with lbm_sw.Batch(sizes, stream=torch_stream(), temporal_steps=temporal) as batch:
            for i, W0 in enumerate(states):
                batch.set_state(i, *W0)
            if temporal == 0:
                t = batch.autotune(2)
                assert t.candidates == 16 + 3 and t.temporal_steps in (1, 4, 6, 8)
            batch.step(30)
            out.append([batch.populations(i) for i in (0, 7, 19, 47)])
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_batch_temporal_needs_fp32_and_even_k_with_boundaries():
    with pytest.raises(lbm_sw.LbmSwError):
        lbm_sw.Batch([(32, 32)], bc=(W, W, P, P), stream=torch_stream(), temporal_steps=5)
    with pytest.raises(lbm_sw.LbmSwError):
        lbm_sw.Batch([(32, 32)], precision=lbm_sw.FP64, stream=torch_stream(), temporal_steps=4)
    with lbm_sw.Batch([(32, 32)], bc=(W, W, P, P), stream=torch_stream()) as batch:
        assert batch.tuning().temporal_steps == 6
    with lbm_sw.Batch([(32, 32)], precision=lbm_sw.FP64, stream=torch_stream()) as batch:
        assert batch.tuning().temporal_steps == 1  # FP64 keeps one step per launch


@pytest.mark.parametrize("bc", [(W, W, W, W), (W, O, I, W), (I, W, P, P), (P, P, W, O)],
                         ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("k", [2, 4, 6, 8])
def test_batch_temporal_with_boundaries(k, bc):
    """Walls, inflow and outflow shared by the batch's instances: the two-column wavefront with
    the side rules over the work list against one tile-list launch per step, bit for bit, on
    odd and even sizes, instances narrower than a strip and wider than several."""
    sizes = [(1, 1), (2, 3), (7, 5), (64, 64), (130, 9), (257, 33), (100, 200), (513, 3), (400, 37)]
    states = _states(sizes, seed=1400 + k)
    out = []
    for temporal in (1, k):
        with lbm_sw.Batch(sizes, bc=bc, inflow=INFLOW, stream=torch_stream(), temporal_steps=temporal) as batch:
            for i, W0 in enumerate(states):
                batch.set_state(i, *W0)
            batch.step(2 * k + 3)
            assert batch.tuning().temporal_steps == temporal
            out.append([batch.populations(i) for i in range(len(sizes))])
    for i in range(len(sizes)):
        assert np.array_equal(out[0][i], out[1][i]), (k, sizes[i])
