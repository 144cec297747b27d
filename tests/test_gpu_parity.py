"""GPU (C ABI) against the oracle, element by element, on tiny and ragged grids.

Every case starts from the same seeded, non-equilibrium pre-collision populations
on both sides (rounded to FP32 first for FP32 runs), runs a few fused steps and
compares the post-collision populations.  The grids cover single cells, odd and
even sizes, several warps per row with ragged tails (a warp spans 128 FP32 or 64
FP64 cells), every boundary kind on every side, and both step kernels.
"""

import numpy as np
import pytest

from paper_1401_0427_gb300 import inputs, lbm_sw

from gpu_helpers import FP32_ELEM_TOL, FP64_TOL, gpu_post, oracle_params, oracle_post, rel_max

pytestmark = pytest.mark.gpu

P, W, O, I = lbm_sw.PERIODIC, lbm_sw.WALL, lbm_sw.OUTFLOW, lbm_sw.INFLOW
INFLOW_STATES = [(1.3, 0.2, -0.1), (0.9, -0.15, 0.05), (1.1, 0.05, 0.12), (1.2, -0.08, -0.2)]

SIZES = [(1, 1), (2, 1), (1, 2), (3, 2), (5, 7), (7, 5), (8, 3), (33, 17), (64, 4), (130, 9), (257, 3)]
BCS = [(P, P, P, P), (W, W, W, W), (O, O, O, O), (I, I, I, I), (I, W, P, P), (P, P, W, O), (W, O, I, W),
       (O, I, W, I)]


def _case(nx, ny, bc, steps, precision, kernel, seed):
    F0 = inputs.random_populations(13, ny, nx, seed=seed)
    if precision == lbm_sw.FP32:
        F0 = F0.astype(np.float32).astype(np.float64)
    got = gpu_post(F0, steps, dim=2, precision=precision, bc=bc, inflow=INFLOW_STATES, a=0.05, kernel=kernel)
    p = oracle_params(nx, ny, 2, bc, INFLOW_STATES, 0.05)
    want = oracle_post(F0, steps, p, 2)
    return rel_max(got, want)


@pytest.mark.parametrize("kernel", [lbm_sw.KERNEL_SIMPLE, lbm_sw.KERNEL_VEC])
@pytest.mark.parametrize("bc", BCS, ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("nx,ny", SIZES)
def test_2d_fp64_matches_oracle(nx, ny, bc, kernel):
    for steps in (1, 4):
        err = _case(nx, ny, bc, steps, lbm_sw.FP64, kernel, seed=1000 + nx * 37 + ny)
        assert err <= FP64_TOL, (steps, err)


@pytest.mark.parametrize("kernel", [lbm_sw.KERNEL_SIMPLE, lbm_sw.KERNEL_VEC])
@pytest.mark.parametrize("bc", BCS, ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("nx,ny", SIZES)
def test_2d_fp32_matches_oracle(nx, ny, bc, kernel):
    for steps in (1, 4):
        err = _case(nx, ny, bc, steps, lbm_sw.FP32, kernel, seed=2000 + nx * 37 + ny)
        assert err <= FP32_ELEM_TOL, (steps, err)


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
@pytest.mark.parametrize("bc", [(P, P), (W, W), (O, O), (I, I), (W, O), (I, W)], ids=str)
@pytest.mark.parametrize("n", [1, 2, 3, 31, 129, 1000])
def test_1d_matches_oracle(n, bc, precision):
    inflow = [(1.3, 0.2, 0.0), (0.9, -0.15, 0.0), None, None]
    for steps in (1, 5):
        F0 = inputs.random_populations(5, 1, n, seed=3000 + n)
        if precision == lbm_sw.FP32:
            F0 = F0.astype(np.float32).astype(np.float64)
        got = gpu_post(F0, steps, dim=1, precision=precision, bc=bc, inflow=inflow, a=0.15)
        want = oracle_post(F0, steps, oracle_params(n, 1, 1, bc, inflow, 0.15), 1)
        err = rel_max(got, want)
        assert err <= (FP64_TOL if precision == lbm_sw.FP64 else FP32_ELEM_TOL), (steps, err)


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
@pytest.mark.parametrize("bc", [(P, P), (W, W), (O, I), (I, W)], ids=str)
@pytest.mark.parametrize("n", [1, 2, 5, 17, 64, 65, 130, 1000, 4097, 16384, 16385])
@pytest.mark.parametrize("steps", [1, 8, 23])
def test_1d_cluster_kernel_equals_per_step_kernel(n, bc, precision, steps):
    """All steps in one cluster launch (the line in shared memory, blocks of 8 steps per
    cluster barrier) against one launch per step: the same arithmetic, so the same bits;
    lines longer than the cluster holds fall back to the per-step kernel."""
    inflow = [(1.3, 0.2, 0.0), (0.9, -0.15, 0.0), None, None]
    F0 = inputs.random_populations(5, 1, n, seed=3500 + n)
    a = gpu_post(F0, steps, dim=1, precision=precision, bc=bc, inflow=inflow, a=0.15, kernel=lbm_sw.KERNEL_SIMPLE)
    b = gpu_post(F0, steps, dim=1, precision=precision, bc=bc, inflow=inflow, a=0.15, kernel=lbm_sw.KERNEL_CLUSTER)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
def test_kernel_variants_are_bitwise_identical(precision):
    """Both step kernels evaluate the same explicitly rounded operations."""
    for (nx, ny), bc in [((257, 19), (I, W, P, P)), ((130, 33), (W, O, I, W)), ((64, 64), (P, P, P, P))]:
        F0 = inputs.random_populations(13, ny, nx, seed=4000 + nx)
        a = gpu_post(F0, 6, dim=2, precision=precision, bc=bc, inflow=INFLOW_STATES, a=0.05,
                     kernel=lbm_sw.KERNEL_SIMPLE)
        b = gpu_post(F0, 6, dim=2, precision=precision, bc=bc, inflow=INFLOW_STATES, a=0.05,
                     kernel=lbm_sw.KERNEL_VEC)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
def test_graph_replay_equals_single_launches(precision):
    F0 = inputs.random_populations(13, 40, 70, seed=5000)
    a = gpu_post(F0, 70, dim=2, precision=precision, bc=(W, O, P, P), inflow=INFLOW_STATES, a=0.05, graph_chunk=-1)
    b = gpu_post(F0, 70, dim=2, precision=precision, bc=(W, O, P, P), inflow=INFLOW_STATES, a=0.05, graph_chunk=16)
    assert np.array_equal(a, b)
