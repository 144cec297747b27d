"""The schemes at a = 0: GPU (C ABI) against the oracle through every kernel family.

With a = 0 the rest potential h_0^* = (a/2) K theta^2 vanishes (section 2,
Eq. 2-potentiels-st-venant-1d; section 3, the 2D potentials), so the rest equilibrium
f_0^eq = a K theta is 0.  Started with f_0 = 0 (an equilibrium state, or populations whose
f_0 plane is zero), the rest population is relaxed towards 0 from 0 and never streams, so
it stays exactly 0: D1Q3Q2 reduces to D1Q2 per conserved component (h, hu) and D2Q5Q4Q4 to
D2Q4 per component (h, hu, hv).  These are the lattices the workloads name.

Cases: one step per launch (SIMPLE and VEC, FP64 and FP32, ragged grids, every boundary
kind), the fused temporal kernels at K = 4 and 6 (FP32; against the oracle and bit for bit
against one step per launch), the 1D cluster kernel, and the shock-tube and dam-break
workloads over their whole runs.  Bars: FP64 max |gpu - oracle| / max |oracle| <= 1e-12;
FP32 element-wise <= 1e-5 of the field scale for runs of a few steps and relative L1 of h
<= 1e-5 for whole runs.  f_0 must be exactly 0 on the GPU after every run.
"""

import numpy as np
import pytest

import oracle
from paper_1401_0427_gb300 import inputs, lbm_sw

from gpu_helpers import FP32_ELEM_TOL, FP32_L1_TOL, FP64_TOL, oracle_params, oracle_post, rel_l1, rel_max, \
    torch_stream

pytestmark = pytest.mark.gpu

P, W, O, I = lbm_sw.PERIODIC, lbm_sw.WALL, lbm_sw.OUTFLOW, lbm_sw.INFLOW
INFLOW = [(1.3, 0.2, -0.1), (0.9, -0.15, 0.05), (1.1, 0.05, 0.12), (1.2, -0.08, -0.2)]
BCS = [(P, P, P, P), (W, W, W, W), (I, W, P, P), (W, O, I, W), (O, I, W, O)]


def _populations_without_rest(q, ny, nx, seed, precision):
    F0 = inputs.random_populations(q, ny, nx, seed=seed)
    F0[0] = 0.0
    if precision == lbm_sw.FP32:
        F0 = F0.astype(np.float32).astype(np.float64)
    return F0


def _gpu(F0, steps, *, dim, precision, bc, kernel, k=0):
    q, ny, nx = F0.shape
    with lbm_sw.Simulation(nx, ny, dim=dim, precision=precision, bc=bc, inflow=INFLOW, a=0.0, kernel=kernel,
                           temporal_steps=k, stream=torch_stream()) as sim:
        sim.set_populations(F0, form=lbm_sw.PRE_COLLISION)
        sim.step(steps)
        return sim.populations().astype(np.float64)


def _tol(precision):
    return FP64_TOL if precision == lbm_sw.FP64 else FP32_ELEM_TOL


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
@pytest.mark.parametrize("kernel", [lbm_sw.KERNEL_SIMPLE, lbm_sw.KERNEL_VEC])
@pytest.mark.parametrize("bc", BCS, ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 2), (7, 5), (33, 17), (130, 9), (257, 3)])
def test_2d_one_step_kernels_at_a0_match_oracle(nx, ny, bc, kernel, precision):
    F0 = _populations_without_rest(13, ny, nx, 8000 + nx * 31 + ny, precision)
    p = oracle_params(nx, ny, 2, bc, INFLOW, 0.0)
    for steps in (1, 4):
        got = _gpu(F0, steps, dim=2, precision=precision, bc=bc, kernel=kernel)
        want = oracle_post(F0, steps, p, 2)
        assert np.all(want[0] == 0.0)  # the oracle's rest population stays 0 as well
        assert np.all(got[0] == 0.0), steps
        assert rel_max(got, want) <= _tol(precision), steps


@pytest.mark.parametrize("k", [4, 6])
@pytest.mark.parametrize("bc", BCS, ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("nx,ny", [(64, 9), (257, 33), (300, 40), (490, 17)])
def test_2d_temporal_kernels_at_a0_match_oracle(nx, ny, bc, k):
    """K fused steps per launch (the two-column wavefront, FP32) at a = 0: against the oracle
    after one launch, and bit for bit against one step per launch over several launches."""
    F0 = _populations_without_rest(13, ny, nx, 8300 + nx + ny + k, lbm_sw.FP32)
    got = _gpu(F0, k, dim=2, precision=lbm_sw.FP32, bc=bc, kernel=lbm_sw.KERNEL_TEMPORAL, k=k)
    want = oracle_post(F0, k, oracle_params(nx, ny, 2, bc, INFLOW, 0.0), 2)
    assert np.all(got[0] == 0.0)
    assert rel_max(got, want) <= FP32_ELEM_TOL
    fused = _gpu(F0, 3 * k + 1, dim=2, precision=lbm_sw.FP32, bc=bc, kernel=lbm_sw.KERNEL_TEMPORAL, k=k)
    single = _gpu(F0, 3 * k + 1, dim=2, precision=lbm_sw.FP32, bc=bc, kernel=lbm_sw.KERNEL_VEC)
    assert np.array_equal(fused, single) and np.all(fused[0] == 0.0)


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
@pytest.mark.parametrize("bc", [(P, P), (W, W), (O, I), (I, W)], ids=str)
@pytest.mark.parametrize("n", [1, 2, 17, 130, 1000, 4097])
def test_1d_cluster_kernel_at_a0_matches_oracle(n, bc, precision):
    F0 = _populations_without_rest(5, 1, n, 8600 + n, precision)
    p = oracle_params(n, 1, 1, bc, INFLOW, 0.0)
    for steps in ((1, 8, 23) if precision == lbm_sw.FP64 else (1, 5)):
        got = _gpu(F0, steps, dim=1, precision=precision, bc=bc, kernel=lbm_sw.KERNEL_CLUSTER)
        want = oracle_post(F0, steps, p, 1)
        assert np.all(got[0] == 0.0), steps
        assert rel_max(got, want) <= _tol(precision), steps


def _run_workload(nx, ny, W0, steps, *, dim, precision, bc, inflow=None):
    with lbm_sw.Simulation(nx, ny, dim=dim, precision=precision, bc=bc, inflow=inflow, a=0.0,
                           stream=torch_stream()) as sim:
        sim.set_state(*W0)
        sim.step(steps)
        return sim.moments(), sim.populations()


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
def test_shock_tube_1000_at_a0(precision):
    """The 1D dam-break workload on the D1Q2-per-component lattice: 1000 cells, h = 2 | 1,
    walls, 500 steps."""
    n, steps = 1000, 500
    h, q = inputs.dam_break_1d(n)
    p = oracle.params(n, a=0.0, bc=(oracle.WALL, oracle.WALL))
    F = oracle.run_1d(oracle.equilibrium_1d(h, q, p), steps, p)
    assert np.all(F[0] == 0.0)
    oh, oq = oracle.moments_1d(F, p)
    (gh, gq), pops = _run_workload(n, 1, (h, q), steps, dim=1, precision=precision, bc=(W, W))
    assert np.all(pops[0] == 0.0)
    if precision == lbm_sw.FP64:
        assert rel_max(gh, oh) <= FP64_TOL and np.abs(gq - oq).max() <= FP64_TOL * np.abs(oh).max()
    else:
        assert rel_l1(gh, oh) <= FP32_L1_TOL


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
def test_dam_break_1024_at_a0(precision):
    """The circular dam-break on the D2Q4-per-component lattice, 1024^2 periodic, 250 steps
    (in FP32 the fused kernel, 6 steps per launch)."""
    n, steps = 1024, 250
    W0 = inputs.circular_dam_break_2d(n, seed=inputs.stream_seed(3, 1024))
    p = oracle.params(n, n, a=0.0)
    F = oracle.run_2d(oracle.equilibrium_2d(*W0, p), steps, p)
    assert np.all(F[0] == 0.0)
    oh, ohu, ohv = oracle.moments_2d(F, p)
    (gh, ghu, ghv), pops = _run_workload(n, n, W0, steps, dim=2, precision=precision, bc=(P, P, P, P))
    assert np.all(pops[0] == 0.0)
    if precision == lbm_sw.FP64:
        assert rel_max(gh, oh) <= FP64_TOL
        assert max(np.abs(ghu - ohu).max(), np.abs(ghv - ohv).max()) <= FP64_TOL * np.abs(oh).max()
    else:
        assert rel_l1(gh, oh) <= FP32_L1_TOL
