"""Temporal blocking (K = 2 .. 8 fused steps per launch through shared memory) against the
one-step-per-launch kernel: every cell update is the same pull + collide, so the results
must be equal bit for bit, on ragged grids (even K takes the kernel that updates two columns
per thread with paired FP32 instructions, 256 - 2K or 192 - 2K output columns per strip, at
K = 6 with the input row's non-shifting planes in registers; odd K a strip of 192 - 2K
columns on all-periodic domains, 128 - 2K otherwise), with every boundary kind, for step
counts that leave a remainder, and on the 4096^2 dam-break."""

import numpy as np
import pytest

from paper_1401_0427_gb300 import inputs, lbm_sw

from gpu_helpers import torch_stream

pytestmark = pytest.mark.gpu

P, W, O, I = lbm_sw.PERIODIC, lbm_sw.WALL, lbm_sw.OUTFLOW, lbm_sw.INFLOW
INFLOW = [(1.3, 0.2, -0.1), (0.9, -0.15, 0.05), (1.1, 0.05, 0.12), (1.2, -0.08, -0.2)]


def _run(F0, steps, bc, kernel, k=0):
    q, ny, nx = F0.shape
    with lbm_sw.Simulation(nx, ny, precision=lbm_sw.FP32, bc=bc, inflow=INFLOW, kernel=kernel, temporal_steps=k,
                           stream=torch_stream()) as sim:
        sim.set_populations(F0, form=lbm_sw.PRE_COLLISION)
        sim.step(steps)
        return sim.populations()


@pytest.mark.parametrize("bc", [(P, P, P, P), (W, W, W, W), (W, O, I, W), (I, W, P, P), (O, I, W, O), (P, P, W, O)],
                         ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 2), (7, 5), (64, 9), (119, 17), (120, 3), (121, 40), (241, 33),
                                   (300, 1), (5, 300), (513, 70)])
@pytest.mark.parametrize("k", [2, 3, 4, 5, 6, 7, 8])
def test_temporal_equals_single_steps(nx, ny, bc, k):
    F0 = inputs.random_populations(13, ny, nx, seed=7000 + nx * 3 + ny).astype(np.float32)
    for steps in (1, 4, 9, 13):
        a = _run(F0, steps, bc, lbm_sw.KERNEL_VEC)
        b = _run(F0, steps, bc, lbm_sw.KERNEL_TEMPORAL, k)
        assert np.array_equal(a, b), (steps, nx, ny)


def test_temporal_equals_single_steps_on_the_benchmark_workload():
    n = 4096
    W0 = inputs.circular_dam_break_2d(n, seed=inputs.stream_seed(3))
    out = []
    for kernel in (lbm_sw.KERNEL_VEC, lbm_sw.KERNEL_TEMPORAL):
        with lbm_sw.Simulation(n, n, precision=lbm_sw.FP32, kernel=kernel, stream=torch_stream()) as sim:
            sim.set_state(*W0)
            sim.step(1000)
            out.append(sim.moments()[0])
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("nx,ny,bc,precision,want", [
    (1024, 1024, (P, P, P, P), lbm_sw.FP32, lbm_sw.KERNEL_TEMPORAL),
    (2048, 512, (P, P, P, P), lbm_sw.FP32, lbm_sw.KERNEL_TEMPORAL),
    (1024, 1024, (W, W, W, W), lbm_sw.FP32, lbm_sw.KERNEL_TEMPORAL),
    (2048, 1024, (I, O, W, W), lbm_sw.FP32, lbm_sw.KERNEL_TEMPORAL),
    (1023, 1040, (W, W, W, W), lbm_sw.FP32, lbm_sw.KERNEL_TEMPORAL),
    (1023, 1040, (P, P, P, P), lbm_sw.FP32, lbm_sw.KERNEL_TEMPORAL),
    (1023, 1040, (P, P, W, O), lbm_sw.FP32, lbm_sw.KERNEL_TEMPORAL),
    (1024, 1024, (P, P, P, P), lbm_sw.FP64, lbm_sw.KERNEL_VEC),
    (512, 512, (P, P, P, P), lbm_sw.FP32, lbm_sw.KERNEL_VEC),
    (512, 512, (I, W, P, P), lbm_sw.FP32, lbm_sw.KERNEL_VEC),
    (627, 627, (P, P, P, P), lbm_sw.FP32, lbm_sw.KERNEL_VEC),
    (628, 628, (P, P, P, P), lbm_sw.FP32, lbm_sw.KERNEL_TEMPORAL),
    (724, 724, (I, W, P, P), lbm_sw.FP32, lbm_sw.KERNEL_TEMPORAL),
    (640, 640, (P, P, P, P), lbm_sw.FP64, lbm_sw.KERNEL_VEC),
])
def test_auto_kernel_choice(nx, ny, bc, precision, want):
    """Temporal blocking from 3 * 2^17 cells (628^2 and up) for FP32; FP64 steps one per launch."""
    with lbm_sw.Simulation(nx, ny, precision=precision, bc=bc, inflow=INFLOW, stream=torch_stream()) as sim:
        assert sim.info().kernel == want


@pytest.mark.parametrize("nx,ny,want", [(628, 628, 4), (1023, 1024, 4), (1024, 1024, 6), (4096, 256, 6)])
def test_default_steps_per_launch(nx, ny, want):
    """The default fused steps per launch: 4 below 2^20 cells, 6 from there."""
    with lbm_sw.Simulation(nx, ny, stream=torch_stream()) as sim:
        assert sim.info().steps_per_launch == want
    with lbm_sw.Simulation(nx, ny, kernel=lbm_sw.KERNEL_TEMPORAL, bc=(W, W, W, W), stream=torch_stream()) as sim:
        assert sim.info().steps_per_launch == want


# Launches of lbm_sw_step(n) at K = 6: launches of 6 while more than 14 steps remain, then the
# cheapest split of the rest into fused launches (4 + 4 in place of 6 + 2; odd sizes only on
# periodic BGK grids, else one single step for an odd count).
SCHEDULES_PERIODIC = {1: 1, 2: 1, 3: 1, 4: 1, 5: 1, 6: 1, 7: 2, 8: 2, 9: 2, 10: 2, 12: 2, 13: 3, 14: 3, 20: 4, 22: 4,
                      23: 4, 1000: 167}
SCHEDULES_WALLS = {1: 1, 2: 1, 3: 2, 5: 2, 7: 2, 8: 2, 13: 3, 20: 4, 22: 4, 23: 5}


@pytest.mark.parametrize("steps", sorted(SCHEDULES_PERIODIC))
def test_auto_temporal_counts_launches_and_steps(steps):
    """AUTO on a periodic 1024^2 FP32 grid: 6 steps per launch, the tail split into fused
    launches (20 = 6 + 6 + 4 + 4, 22 = 6 + 6 + 6 + 4, 8 = 4 + 4)."""
    W0 = inputs.circular_dam_break_2d(1024, seed=inputs.stream_seed(3))
    with lbm_sw.Simulation(1024, 1024, stream=torch_stream()) as sim:
        sim.set_state(*W0)
        before = sim.info().kernel_launches
        sim.step(steps)
        info = sim.info()
        assert info.steps_done == steps and info.steps_per_launch == 6
        assert info.kernel_launches - before == SCHEDULES_PERIODIC[steps]


@pytest.mark.parametrize("bc", [(P, P, P, P), (W, W, W, W), (I, O, W, W)], ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("steps", [2, 3, 5, 7, 8, 13, 20, 22, 23])
def test_mixed_schedule_equals_single_steps(bc, steps):
    """The split tails (fused launches of 2 .. 6 steps, a single step only for an odd count on
    sides that are not periodic) give the bits of one step per launch."""
    n = 1024
    F0 = inputs.random_populations(13, 96, n, seed=7700 + steps).astype(np.float32)
    F0 = np.ascontiguousarray(np.tile(F0, (1, n // 96 + 1, 1))[:, :n, :])
    a = _run(F0, steps, bc, lbm_sw.KERNEL_VEC)
    with lbm_sw.Simulation(n, n, precision=lbm_sw.FP32, bc=bc, inflow=INFLOW, stream=torch_stream()) as sim:
        assert sim.info().kernel == lbm_sw.KERNEL_TEMPORAL and sim.info().steps_per_launch == 6
        sim.set_populations(F0, form=lbm_sw.PRE_COLLISION)
        before = sim.info().kernel_launches
        sim.step(steps)
        launches = sim.info().kernel_launches - before
        b = sim.populations()
    assert np.array_equal(a, b), steps
    if bc != (P, P, P, P):
        assert launches == SCHEDULES_WALLS[steps]


@pytest.mark.parametrize("bc", [(P, P, P, P), (W, W, W, W), (W, O, I, W), (I, W, P, P), (O, I, W, O), (P, P, W, O)],
                         ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("nx,ny", [(2, 3), (4, 4), (10, 7), (244, 5), (246, 9), (488, 20), (490, 33), (1024, 130),
                                   (3, 4), (245, 9), (247, 6), (489, 20), (1023, 17)])
@pytest.mark.parametrize("k", [2, 4, 6, 8])
def test_paired_kernel_equals_single_steps(nx, ny, k, bc):
    """Widths around the strip width (256 - 2K up to K = 6, 192 - 2K at K = 8), where the
    paired kernel runs, with every boundary kind (a width of 2 puts both x sides in one pair;
    an odd width puts the last column in the first lane of a pair, and with periodic x sides
    the pairs across the seam land in two copies)."""
    F0 = inputs.random_populations(13, ny, nx, seed=7500 + nx + ny).astype(np.float32)
    for steps in (k, 3 * k + 1):
        a = _run(F0, steps, bc, lbm_sw.KERNEL_VEC)
        b = _run(F0, steps, bc, lbm_sw.KERNEL_TEMPORAL, k)
        assert np.array_equal(a, b), (steps, nx, ny)


@pytest.mark.parametrize("bc", [(W, W, W, W), (I, O, W, W)], ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("steps", [2, 20])
def test_large_bounded_kernel_equals_single_steps(bc, steps):
    """Grids of 2^21 cells or more with walls, inflow and outflow run the two-column
    wavefront in 256-column strips (K = 6, and K = 4 and 2 for the tails, with the input
    row's f0 and +y movers in registers): bit for bit equal to one step per launch."""
    nx, ny = 2900, 2900
    tile = inputs.random_populations(13, 96, nx, seed=8100 + steps).astype(np.float32)
    F0 = np.ascontiguousarray(np.tile(tile, (1, ny // 96 + 1, 1))[:, :ny, :])
    a = _run(F0, steps, bc, lbm_sw.KERNEL_VEC)
    with lbm_sw.Simulation(nx, ny, precision=lbm_sw.FP32, bc=bc, inflow=INFLOW, stream=torch_stream()) as sim:
        assert sim.info().kernel == lbm_sw.KERNEL_TEMPORAL and sim.info().steps_per_launch == 6
        sim.set_populations(F0, form=lbm_sw.PRE_COLLISION)
        sim.step(steps)
        b = sim.populations()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("nx,ny,steps", [(2900, 2900, 2), (2900, 2900, 3), (2900, 2900, 5), (2900, 2900, 6),
                                         (2900, 2900, 11), (2900, 2900, 13), (2900, 2900, 20), (3002, 2795, 20),
                                         (2901, 2901, 5), (2901, 2901, 20)])
def test_large_periodic_kernel_equals_single_steps(nx, ny, steps):
    """Periodic grids of 2^23 cells or more with an even width run K = 6 in 256-column
    strips (the headline kernel, with its branch-free steady state), and their tails K = 4,
    2, and the odd K = 5 and 3 (paired with an even left halo: 20 = 6 + 6 + 4 + 4, 11 = 6 + 5,
    2, 3, 5), and the odd-width form (2901): bit for bit equal to one step per launch on non-equilibrium populations (a seeded random 96-row tile repeated over
    the grid; 3002 x 2795 has a narrow last strip and an odd height)."""
    tile = inputs.random_populations(13, 96, nx, seed=7900 + steps + nx).astype(np.float32)
    F0 = np.ascontiguousarray(np.tile(tile, (1, ny // 96 + 1, 1))[:, :ny, :])
    a = _run(F0, steps, (P, P, P, P), lbm_sw.KERNEL_VEC)
    with lbm_sw.Simulation(nx, ny, precision=lbm_sw.FP32, stream=torch_stream()) as sim:
        assert sim.info().kernel == lbm_sw.KERNEL_TEMPORAL and sim.info().steps_per_launch == 6
        sim.set_populations(F0, form=lbm_sw.PRE_COLLISION)
        sim.step(steps)
        b = sim.populations()
    assert np.array_equal(a, b)
