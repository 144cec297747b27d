"""Obstacles (solid cells with mirror walls on their faces) on the GPU against the oracle.

The oracle's obstacle rule is pinned to its domain-side wall in test_oracle_obstacles.py.
Here the obstacle kernel matches the oracle element by element on random masks with every
boundary kind, in FP64 (1e-12) and FP32 (1e-5 of the field scale); with an empty mask it
equals the SIMPLE kernel bit for bit; graph replay, removal of the mask, the solid cells'
populations and the adjoint's refusal are checked; and Emery's forward-facing step of
section 4 (lambda = 80, Froude 3) equals the oracle's run on the paper's coarse mesh.
"""

import numpy as np
import pytest

import oracle
from paper_1401_0427_gb300 import experiments as ex
from paper_1401_0427_gb300 import inputs, lbm_sw

from gpu_helpers import FP32_ELEM_TOL, FP64_TOL, gpu_post, oracle_params, oracle_post, rel_max, torch_stream

pytestmark = pytest.mark.gpu

P, W, O, I = lbm_sw.PERIODIC, lbm_sw.WALL, lbm_sw.OUTFLOW, lbm_sw.INFLOW
INFLOW_STATES = [(1.3, 0.2, -0.1), (0.9, -0.15, 0.05), (1.1, 0.05, 0.12), (1.2, -0.08, -0.2)]
SIZES = [(1, 1), (3, 2), (7, 5), (33, 17), (64, 9), (130, 12)]
BCS = [(P, P, P, P), (W, W, W, W), (O, O, O, O), (I, I, I, I), (I, O, W, W), (P, P, W, O)]


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
@pytest.mark.parametrize("bc", BCS, ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("nx,ny", SIZES)
def test_obstacles_match_oracle(nx, ny, bc, precision):
    solid = inputs.random_obstacles(ny, nx, seed=900 + nx * 7 + ny, fraction=0.25)
    F0 = inputs.random_populations(13, ny, nx, seed=910 + nx * 7 + ny)
    if precision == lbm_sw.FP32:
        F0 = F0.astype(np.float32).astype(np.float64)
    p = oracle_params(nx, ny, 2, bc, INFLOW_STATES, 0.05, solid=solid)
    for steps in (1, 5):
        got = gpu_post(F0, steps, dim=2, precision=precision, bc=bc, inflow=INFLOW_STATES, a=0.05, solid=solid)
        want = oracle_post(F0, steps, p, 2)
        assert rel_max(got, want) <= (FP64_TOL if precision == lbm_sw.FP64 else FP32_ELEM_TOL), steps
        assert np.array_equal(got[:, solid != 0], F0[:, solid != 0])  # solid cells keep their populations


@pytest.mark.parametrize("mrt", [False, True], ids=["bgk", "mrt"])
@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
@pytest.mark.parametrize("bc", BCS, ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("nx,ny,fraction", [(1, 1, 0.5), (3, 2, 0.3), (7, 5, 0.3), (33, 17, 0.05), (130, 12, 0.25),
                                            (257, 33, 0.02), (513, 20, 0.3), (129, 64, 0.0)])
def test_vectorised_obstacle_kernel_equals_one_thread_per_cell(nx, ny, fraction, bc, precision, mrt):
    """The row kernel (16-byte vectors, warp shuffles, a warp with no solid cell near it on the
    plain path) against the one-thread-per-cell obstacle kernel: the same operations on the
    same values, so the same bits, over several steps."""
    solid = inputs.random_obstacles(ny, nx, seed=930 + nx + ny, fraction=fraction)
    F0 = inputs.random_populations(13, ny, nx, seed=940 + nx + ny)
    rates = [0.0, 1.1, 1.2, 1.3, 1.4, 0.0, 1.5, 1.6, 1.7, 0.0, 1.75, 1.65, 0.9] if mrt else None
    kw = dict(dim=2, precision=precision, bc=bc, inflow=INFLOW_STATES, a=0.05, solid=solid, mrt_rates=rates)
    a = gpu_post(F0, 7, kernel=lbm_sw.KERNEL_SIMPLE, **kw)
    b = gpu_post(F0, 7, kernel=lbm_sw.KERNEL_VEC, **kw)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
def test_empty_mask_equals_simple_kernel(precision):
    F0 = inputs.random_populations(13, 19, 70, seed=920)
    kw = dict(dim=2, precision=precision, bc=(I, W, P, P), inflow=INFLOW_STATES, a=0.05)
    a = gpu_post(F0, 9, kernel=lbm_sw.KERNEL_SIMPLE, **kw)
    b = gpu_post(F0, 9, solid=np.zeros((19, 70), dtype=np.uint8), **kw)
    assert np.array_equal(a, b)


def test_graph_replay_removal_and_temporal_default():
    n = 1024
    solid = np.zeros((n, n), dtype=np.uint8)
    solid[400:600, 300:340] = 1
    W0 = inputs.circular_dam_break_2d(n, seed=inputs.stream_seed(3))
    out = []
    for graph_chunk in (-1, 16):
        with lbm_sw.Simulation(n, n, stream=torch_stream(), graph_chunk=graph_chunk) as sim:
            assert sim.info().kernel == lbm_sw.KERNEL_TEMPORAL and sim.info().steps_per_launch == 6
            sim.set_state(*W0)
            sim.set_obstacle(solid)
            assert sim.info().steps_per_launch == 1
            sim.step(40)
            out.append(sim.populations())
            sim.set_obstacle(None)
            assert sim.info().steps_per_launch == 6
            sim.step(12)
            out.append(sim.populations())
    assert np.array_equal(out[0], out[2]) and np.array_equal(out[1], out[3])
    with lbm_sw.Simulation(n, n, stream=torch_stream(), kernel=lbm_sw.KERNEL_SIMPLE) as sim:
        sim.set_state(*W0)
        sim.set_obstacle(solid)
        sim.step(40)
        assert np.array_equal(sim.populations(), out[0])


def test_device_mask_and_errors():
    import torch

    nx, ny = 40, 30
    solid = inputs.random_obstacles(ny, nx, seed=930)
    F0 = inputs.random_populations(13, ny, nx, seed=931)
    host = gpu_post(F0, 6, dim=2, precision=lbm_sw.FP64, bc=(W, W, W, W), inflow=None, a=0.05, solid=solid)
    with lbm_sw.Simulation(nx, ny, precision=lbm_sw.FP64, bc=(W, W, W, W), stream=torch_stream()) as sim:
        sim.set_obstacle(torch.from_numpy(solid).cuda())
        sim.set_populations(F0, form=lbm_sw.PRE_COLLISION)
        sim.step(6)
        assert np.array_equal(sim.populations(), host)
        with pytest.raises(lbm_sw.LbmSwError):
            lbm_sw.Tape(sim, 10)
    with lbm_sw.Simulation(100, 1, dim=1, bc=(W, W), stream=torch_stream()) as sim1:
        with pytest.raises(lbm_sw.LbmSwError):
            sim1.set_obstacle(np.zeros((1, 100), dtype=np.uint8))


def test_emery_step_equals_oracle_on_the_coarse_mesh():
    nx, ny = 120, 40
    r = ex.emery_step(nx, ny, t_end=0.5, stream=torch_stream())
    solid, W0, win = inputs.emery_step(nx, ny)
    p = oracle.params(nx, ny, lam=80.0, a=0.05, s=1.8, bc=(oracle.INFLOW, oracle.OUTFLOW, oracle.WALL, oracle.WALL),
                      inflow=[win, None, None, None], solid=solid)
    oh, ou, ov = oracle.moments_2d(oracle.run_2d(oracle.equilibrium_2d(*W0, p), r["steps"], p), p)
    assert rel_max(r["h"], oh) <= FP64_TOL and rel_max(r["hu"], ou) <= FP64_TOL
    # a bow shock stands in front of the step: the depth there exceeds the inflow's
    assert r["max_h"] > 2.5 and r["min_h"] > 0.5
    r32 = ex.emery_step(nx, ny, t_end=0.5, precision=lbm_sw.FP32, stream=torch_stream())
    fluid = solid == 0
    assert np.abs(r32["h"] - r["h"])[fluid].sum() / np.abs(r["h"])[fluid].sum() <= 1e-5


@pytest.mark.parametrize("nx,ny", [(120, 40), (240, 80), (480, 120)])
def test_emery_step_paper_meshes_stay_admissible(nx, ny):
    for t_end in (0.5, 4.0):
        r = ex.emery_step(nx, ny, t_end=t_end, stream=torch_stream())
        fluid = r["solid"] == 0
        assert np.isfinite(r["h"]).all() and r["min_h"] > 0.3 and r["max_h"] < 6.0
        assert np.abs(r["h"][~fluid] - 1.0).max() <= 1e-14  # solid cells keep the initial state
