"""MRT relaxation on the GPU (each moment of the paper's bases at its own rate, Eq.
2-relaxation) against the oracle's MRT collision, which is pinned to the printed moment
definitions (tests/test_oracle_equilibria.py)."""

import numpy as np
import pytest

import oracle
from paper_1401_0427_gb300 import inputs, lbm_sw

from gpu_helpers import FP32_ELEM_TOL, FP64_TOL, gpu_post, oracle_post, rel_max, torch_stream

pytestmark = pytest.mark.gpu

P, W, O, I = lbm_sw.PERIODIC, lbm_sw.WALL, lbm_sw.OUTFLOW, lbm_sw.INFLOW
INFLOW = [(1.3, 0.2, -0.1), (0.9, -0.15, 0.05), (1.1, 0.05, 0.12), (1.2, -0.08, -0.2)]
RATES_2D = [0.0, 1.1, 1.2, 1.3, 1.4, 0.0, 1.5, 1.6, 1.7, 0.0, 1.75, 1.65, 0.9]
RATES_1D = [0.0, 1.3, 1.6, 0.0, 1.9]


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
@pytest.mark.parametrize("kernel", [lbm_sw.KERNEL_SIMPLE, lbm_sw.KERNEL_VEC])
@pytest.mark.parametrize("bc", [(P, P, P, P), (W, O, I, W), (I, W, P, P)], ids=["PPPP", "WOIW", "IWPP"])
@pytest.mark.parametrize("nx,ny", [(1, 1), (5, 7), (130, 9), (257, 3)])
def test_2d_mrt_matches_oracle(nx, ny, bc, kernel, precision):
    F0 = inputs.random_populations(13, ny, nx, seed=6000 + nx)
    if precision == lbm_sw.FP32:
        F0 = F0.astype(np.float32).astype(np.float64)
    p = oracle.params(nx, ny, a=0.05, bc=bc, inflow=INFLOW, s_moments=RATES_2D)
    for steps in (1, 4):
        got = gpu_post(F0, steps, dim=2, precision=precision, bc=bc, inflow=INFLOW, a=0.05, kernel=kernel,
                       mrt_rates=RATES_2D)
        err = rel_max(got, oracle_post(F0, steps, p, 2))
        assert err <= (FP64_TOL if precision == lbm_sw.FP64 else FP32_ELEM_TOL), (steps, err)


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
@pytest.mark.parametrize("kernel", [lbm_sw.KERNEL_SIMPLE, lbm_sw.KERNEL_CLUSTER])
@pytest.mark.parametrize("bc", [(P, P), (W, W), (O, I)], ids=str)
@pytest.mark.parametrize("n", [1, 31, 1000])
def test_1d_mrt_matches_oracle(n, bc, kernel, precision):
    inflow = [(1.3, 0.2, 0.0), (0.9, -0.15, 0.0), None, None]
    F0 = inputs.random_populations(5, 1, n, seed=6100 + n)
    if precision == lbm_sw.FP32:
        F0 = F0.astype(np.float32).astype(np.float64)
    p = oracle.params(n, a=0.15, bc=bc, inflow=inflow, s_moments=RATES_1D)
    for steps in (1, 5):
        got = gpu_post(F0, steps, dim=1, precision=precision, bc=bc, inflow=inflow, a=0.15, kernel=kernel,
                       mrt_rates=RATES_1D)
        err = rel_max(got, oracle_post(F0, steps, p, 1))
        assert err <= (FP64_TOL if precision == lbm_sw.FP64 else FP32_ELEM_TOL), (steps, err)


def test_equal_rates_reproduce_bgk_and_reset():
    F0 = inputs.random_populations(13, 40, 70, seed=6200)
    bgk = gpu_post(F0, 30, dim=2, precision=lbm_sw.FP64, bc=(W, O, P, P), inflow=INFLOW, a=0.05)
    mrt = gpu_post(F0, 30, dim=2, precision=lbm_sw.FP64, bc=(W, O, P, P), inflow=INFLOW, a=0.05,
                   mrt_rates=[1.8] * 13)
    assert rel_max(mrt, bgk) <= 1e-13
    with lbm_sw.Simulation(70, 40, precision=lbm_sw.FP64, bc=(W, O, P, P), inflow=INFLOW, graph_chunk=8,
                           stream=torch_stream()) as sim:
        sim.set_relaxation(RATES_2D)
        sim.set_populations(F0, form=lbm_sw.PRE_COLLISION)
        sim.step(16)  # captures graphs with the MRT constants
        sim.set_relaxation(None)
        sim.step(14)  # the graphs must be rebuilt for BGK
        mixed = sim.populations()
    p_mrt = oracle.params(70, 40, a=0.05, bc=(W, O, P, P), inflow=INFLOW, s_moments=RATES_2D)
    p_bgk = oracle.params(70, 40, a=0.05, bc=(W, O, P, P), inflow=INFLOW)
    F = oracle.run_2d(F0, 16, p_mrt)             # 16 MRT steps from F0 (pre-collision)
    F = oracle.collide_2d(F, p_mrt)              # the state the GPU stores after them
    F = oracle.collide_2d(oracle.run_2d(oracle.stream_2d(F, p_bgk), 13, p_bgk), p_bgk)
    assert rel_max(mixed, F) <= FP64_TOL


def test_mrt_validation_and_adjoint_rejects_mrt():
    with lbm_sw.Simulation(16, 8, stream=torch_stream()) as sim:
        with pytest.raises(lbm_sw.LbmSwError) as ei:
            sim.set_relaxation([1.0] * 5)
        assert "13 rates" in str(ei.value)
        bad = list(RATES_2D)
        bad[3] = 2.5
        with pytest.raises(lbm_sw.LbmSwError):
            sim.set_relaxation(bad)
        sim.set_relaxation(RATES_2D)
        sim.set_state(np.ones((8, 16)), np.zeros((8, 16)), np.zeros((8, 16)))
        with pytest.raises(lbm_sw.LbmSwError) as ei:
            lbm_sw.Tape(sim, 10)
        assert "BGK" in str(ei.value)


def _run_mrt(F0, steps, bc, kernel, k=0):
    q, ny, nx = F0.shape
    with lbm_sw.Simulation(nx, ny, precision=lbm_sw.FP32, bc=bc, inflow=INFLOW, a=0.05, kernel=kernel,
                           temporal_steps=k, stream=torch_stream()) as sim:
        sim.set_relaxation(RATES_2D)
        sim.set_populations(F0, form=lbm_sw.PRE_COLLISION)
        spl = sim.info().steps_per_launch
        sim.step(steps)
        return sim.populations(), spl


@pytest.mark.parametrize("bc", [(P, P, P, P), (W, W, W, W), (W, O, I, W), (I, W, P, P), (P, P, W, O)],
                         ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("nx,ny", [(2, 3), (7, 5), (10, 7), (244, 5), (245, 9), (250, 33), (488, 20), (501, 20),
                                   (1024, 70)])
@pytest.mark.parametrize("k", [2, 4, 6, 8])
def test_mrt_temporal_equals_single_steps(nx, ny, bc, k):
    """FP32 MRT with K steps per launch (the two-column wavefront with collide13x2_mrt) against
    one MRT step per launch: the same rounded operations on the same values, bit for bit."""
    F0 = inputs.random_populations(13, ny, nx, seed=6100 + nx + ny).astype(np.float32)
    for steps in (k, 3 * k + 1):
        a, _ = _run_mrt(F0, steps, bc, lbm_sw.KERNEL_VEC)
        b, spl = _run_mrt(F0, steps, bc, lbm_sw.KERNEL_TEMPORAL, k)
        assert spl == k
        assert np.array_equal(a, b), (steps, nx, ny)


@pytest.mark.parametrize("bc", [(P, P, P, P), (W, O, P, P)], ids=lambda b: "".join("PWOI"[k] for k in b))
def test_mrt_large_grid_temporal_equals_single_steps(bc):
    """Grids of 2^23 cells or more run the MRT wavefront in 256-column strips (periodic: with
    its branch-free steady state): bit for bit equal to one MRT step per launch, 13 steps
    (6 + 6 + 1) on a seeded random 96-row tile repeated over 2900 x 2900 cells."""
    n = 2900
    tile = inputs.random_populations(13, 96, n, seed=6900).astype(np.float32)
    F0 = np.ascontiguousarray(np.tile(tile, (1, n // 96 + 1, 1))[:, :n, :])
    a, _ = _run_mrt(F0, 13, bc, lbm_sw.KERNEL_VEC)
    b, spl = _run_mrt(F0, 13, bc, lbm_sw.KERNEL_AUTO)
    assert spl == 6
    assert np.array_equal(a, b)


def test_mrt_temporal_choice():
    """AUTO on 1024^2 FP32 grids keeps temporal blocking with MRT (the two-column kernel, any
    width and sides)."""
    for nx, bc, want in ((1024, (P, P, P, P), 6), (1024, (W, O, I, W), 6), (1025, (P, P, P, P), 6),
                         (1025, (P, P, W, O), 6), (1025, (W, O, I, W), 6)):
        with lbm_sw.Simulation(nx, 1024, a=0.05, bc=bc, inflow=INFLOW, stream=torch_stream()) as sim:
            sim.set_relaxation(RATES_2D)
            assert sim.info().steps_per_launch == want, (nx, bc)


@pytest.mark.parametrize("n,kernel,bgk,mrt", [(724, lbm_sw.KERNEL_AUTO, 4, 1), (724, lbm_sw.KERNEL_TEMPORAL, 4, 4),
                                               (868, lbm_sw.KERNEL_AUTO, 4, 4)])
def test_mrt_small_grid_choice(n, kernel, bgk, mrt):
    """Below 2^19 cells AUTO steps MRT one step per launch (the BGK collision keeps K = 4),
    while an explicit TEMPORAL choice keeps its fused launches."""
    with lbm_sw.Simulation(n, n, a=0.05, bc=(I, W, P, P), inflow=INFLOW, kernel=kernel, stream=torch_stream()) as sim:
        assert sim.info().steps_per_launch == bgk
        sim.set_relaxation(RATES_2D)
        assert sim.info().steps_per_launch == mrt
        sim.set_relaxation(None)
        assert sim.info().steps_per_launch == bgk


def test_mrt_temporal_matches_oracle():
    F0 = inputs.random_populations(13, 40, 250, seed=6200)
    F0 = F0.astype(np.float32).astype(np.float64)
    bc = (W, O, I, W)
    p = oracle.params(250, 40, a=0.05, bc=bc, inflow=INFLOW, s_moments=RATES_2D)
    want = oracle_post(F0, 12, p, 2)
    got, spl = _run_mrt(F0, 12, bc, lbm_sw.KERNEL_TEMPORAL, 6)
    assert spl == 6
    assert rel_max(got.astype(np.float64), want) <= FP32_ELEM_TOL
