"""Behaviour of the C ABI on the GPU: state round trips, device-pointer transfers,
diagnostics (totals in FP64, NaN / dry-cell detection), error codes, lake at rest."""

import numpy as np
import pytest

import oracle
from paper_1401_0427_gb300 import inputs, lbm_sw

from gpu_helpers import FP64_TOL, torch_stream

pytestmark = pytest.mark.gpu

P, W, O, I = lbm_sw.PERIODIC, lbm_sw.WALL, lbm_sw.OUTFLOW, lbm_sw.INFLOW


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
@pytest.mark.parametrize("bc", [(P, P, P, P), (W, W, W, W), (O, O, O, O), (W, O, P, P)], ids=str)
@pytest.mark.parametrize("h0", [1.0, 2.0, 0.5, 1.37, 0.73, 2.9])
def test_lake_at_rest_stays_at_rest(precision, bc, h0):
    """A lake at rest keeps exactly zero velocities and a uniform depth (every cell rounds
    alike and the x / y mirror pairs cancel exactly).  The BGK step evaluates
    (1 - s) f + s f^eq, which maps the initial equilibrium onto a rounding neighbour: the
    populations settle within about one unit in the last place of it in the first steps and
    stay there (the same bound after 200 and 2000 steps, no drift)."""
    nx, ny = 133, 70
    tol = 1e-14 if precision == lbm_sw.FP64 else 1e-6
    with lbm_sw.Simulation(nx, ny, precision=precision, bc=bc, stream=torch_stream()) as sim:
        sim.set_state(np.full((ny, nx), h0), np.zeros((ny, nx)), np.zeros((ny, nx)))
        F0 = sim.populations().astype(np.float64)
        for n in (200, 1800):
            sim.step(n)
            F = sim.populations().astype(np.float64)
            assert np.abs(F - F0).max() <= tol * np.abs(F0).max()
            h, hu, hv = sim.moments()
            assert np.all(hu == 0) and np.all(hv == 0)
            assert np.all(h == h.flat[0]) and abs(h.flat[0] - h0) <= tol * h0


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
@pytest.mark.parametrize("bc", [(P, P, P, P), (W, O, P, P)], ids=str)
@pytest.mark.parametrize("h0", [1.37, 0.73])
def test_lake_at_rest_is_a_fixed_point_of_the_mrt_collision(precision, bc, h0):
    """The MRT form relaxes f^eq - f, which is exactly zero at rest: with any rates (here all
    equal to s, the BGK operator) the equilibrium maps to itself bit for bit."""
    nx, ny = 133, 70
    with lbm_sw.Simulation(nx, ny, precision=precision, bc=bc, stream=torch_stream()) as sim:
        sim.set_relaxation([0.0] + [1.8] * 4 + [0.0] + [1.8] * 3 + [0.0] + [1.8] * 3)
        sim.set_state(np.full((ny, nx), h0), np.zeros((ny, nx)), np.zeros((ny, nx)))
        F0 = sim.populations()
        W0 = sim.moments()  # the depth of the stored equilibrium (its FP32 sum may round off h0)
        sim.step(200)
        assert np.array_equal(sim.populations(), F0)
        h, hu, hv = sim.moments()
    assert np.array_equal(h, W0[0]) and np.all(h == h.flat[0]) and np.all(hu == 0) and np.all(hv == 0)


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
def test_set_state_is_the_oracle_equilibrium(precision):
    nx, ny = 97, 31
    h, hu, hv = inputs.random_states(nx * ny, seed=77)
    W0 = [x.reshape(ny, nx) for x in (h, hu, hv)]
    with lbm_sw.Simulation(nx, ny, precision=precision, stream=torch_stream()) as sim:
        sim.set_state(*W0)
        F = sim.populations().astype(np.float64)
        m = sim.moments()
    want = oracle.equilibrium_2d(*W0, oracle.params(nx, ny, a=0.05))
    tol = FP64_TOL if precision == lbm_sw.FP64 else 1e-6
    assert np.abs(F - want).max() <= tol * np.abs(want).max()
    for got, w in zip(m, W0):
        assert np.abs(got - w).max() <= tol * np.abs(W0[0]).max()


def test_device_pointers_match_host_path():
    import torch

    nx, ny = 200, 90
    h = np.ascontiguousarray(inputs.circular_dam_break_2d(200, seed=inputs.stream_seed(3))[0][:ny])
    hu = 0.1 * inputs.uniform(5, nx * ny, -1, 1).reshape(ny, nx)
    hv = 0.1 * inputs.uniform(6, nx * ny, -1, 1).reshape(ny, nx)
    with lbm_sw.Simulation(nx, ny, precision=lbm_sw.FP64, bc=(W, W, O, I), inflow=[None, None, None, (1.1, 0, 0.1)],
                           stream=torch_stream()) as a, \
         lbm_sw.Simulation(nx, ny, precision=lbm_sw.FP64, bc=(W, W, O, I), inflow=[None, None, None, (1.1, 0, 0.1)],
                           stream=torch_stream()) as b:
        a.set_state(h, hu, hv)
        b.set_state(*[torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (h, hu, hv)])
        a.step(33)
        b.step(33)
        host = a.moments()
        dev = [torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3)]
        b.moments_into(*dev)
        torch.cuda.synchronize()
        for x, y in zip(host, dev):
            assert np.array_equal(x, y.cpu().numpy())
        Fa = a.populations()
        Fb = torch.empty(Fa.shape, dtype=torch.float64, device="cuda")
        b.populations_into(Fb)
        torch.cuda.synchronize()
        assert np.array_equal(Fa, Fb.cpu().numpy())
        # checkpoint round trip: post-collision populations in, same trajectory out
        b.set_populations(Fb, form=lbm_sw.POST_COLLISION)
        a.step(5)
        b.step(5)
        assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
def test_diagnostics_are_fp64_totals(precision):
    nx, ny = 301, 211
    h, hu, hv = (x.reshape(ny, nx) for x in inputs.random_states(nx * ny, seed=88))
    with lbm_sw.Simulation(nx, ny, precision=precision, bc=(W, W, W, W), stream=torch_stream()) as sim:
        sim.set_state(h, hu, hv)
        sim.step(10)
        m = sim.moments()
        d = sim.diagnostics()
    assert d[4] == lbm_sw.OK
    scale = np.abs(m[0]).sum()
    assert abs(d[0] - m[0].sum()) <= 1e-12 * scale
    assert abs(d[1] - m[1].sum()) <= 1e-12 * scale and abs(d[2] - m[2].sum()) <= 1e-12 * scale
    assert d[3] == m[0].min()


@pytest.mark.parametrize("bc", [(W, W, W, W), (lbm_sw.PERIODIC,) * 4], ids=["walls", "periodic"])
def test_diagnostics_equal_the_oracle_totals(bc):
    """The FP64 diagnostics of the GPU state against the oracle's own moments of its own run
    from the same initial state (not the GPU's moments): sum h, sum hu, sum hv and min h.
    Walls and periodic sides conserve the totals; the run keeps them within rounding of the
    initial totals on both sides."""
    nx, ny, steps = 97, 64, 25
    W0 = [x.reshape(ny, nx) for x in inputs.random_states(nx * ny, seed=89, h=(0.8, 1.4), speed=0.25)]
    with lbm_sw.Simulation(nx, ny, precision=lbm_sw.FP64, bc=bc, stream=torch_stream()) as sim:
        sim.set_state(*W0)
        sim.step(steps)
        d = sim.diagnostics()
    p = oracle.params(nx, ny, a=0.05, bc=bc)
    oh, ohu, ohv = oracle.moments_2d(oracle.run_2d(oracle.equilibrium_2d(*W0, p), steps, p), p)
    scale = np.abs(oh).sum()
    assert d[4] == lbm_sw.OK
    assert abs(d[0] - oh.sum()) <= 1e-12 * scale
    assert abs(d[1] - ohu.sum()) <= 1e-12 * scale and abs(d[2] - ohv.sum()) <= 1e-12 * scale
    assert abs(d[3] - oh.min()) <= 1e-12 * oh.max()
    assert abs(d[0] - W0[0].sum()) <= 1e-12 * scale  # mass conserved by both sides


def test_diagnostics_report_unstable_states():
    nx, ny = 64, 48
    with lbm_sw.Simulation(nx, ny, precision=lbm_sw.FP32, stream=torch_stream()) as sim:
        h = np.ones((ny, nx))
        h[10, 20] = -0.5  # a dry (negative-depth) cell
        sim.set_state(h, np.zeros_like(h), np.zeros_like(h))
        out = sim.diagnostics(raise_unstable=False)
        assert out[4] == lbm_sw.E_UNSTABLE and abs(out[3] + 0.5) < 1e-6
        F = sim.populations()
        F[3, 5, 5] = np.nan
        sim.set_populations(F)
        with pytest.raises(lbm_sw.LbmSwError) as ei:
            sim.diagnostics()
        assert ei.value.status == lbm_sw.E_UNSTABLE and "cells" in str(ei.value)


def test_state_errors_and_counters():
    with lbm_sw.Simulation(40, 30, stream=torch_stream()) as sim:
        with pytest.raises(lbm_sw.LbmSwError) as ei:
            sim.step(1)
        assert ei.value.status == lbm_sw.E_STATE
        with pytest.raises(lbm_sw.LbmSwError) as ei:
            lbm_sw.lbm_sw_step(sim.handle, -1)
        assert ei.value.status == lbm_sw.E_ARG
        sim.set_state(np.ones((30, 40)), np.zeros((30, 40)), np.zeros((30, 40)))
        sim.step(7)
        info = sim.info()
        assert info.q == 13 and info.steps_done == 7 and info.pitch == 64
        assert info.bytes_per_update == 104.0 and info.kernel == lbm_sw.KERNEL_VEC


def test_1d_info():
    with lbm_sw.Simulation(1000, 1, dim=1, precision=lbm_sw.FP64, bc=(W, W), stream=torch_stream()) as sim:
        info = sim.info()
        assert info.q == 5 and info.bytes_per_update == 80.0 and info.kernel == lbm_sw.KERNEL_CLUSTER
