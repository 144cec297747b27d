"""GPU (C ABI) against the oracle on the benchmark workloads.

* 1D dam-break shock tube, 1000 cells, 500 steps, walls: FP64 element-wise, FP32
  relative L1 of h.
* 2D shock reflection, 512 x 512, 2000 steps (inflow x-, wall x+, periodic in y):
  the field is y-invariant (kept bit for bit by both sides), so the oracle runs one
  row of 512 cells and every GPU row is compared with it.
* 2D circular dam-break, 4096 x 4096, 1000 steps: (a) the whole run, FP64 and FP32,
  against the oracle run in full on every host core (marked slow: minutes of
  oracle time), (b) the same physical case at 1024 x 1024 (250 steps, same final
  time) compared in full, (c) at full size, one more step from the GPU state
  recomputed by the oracle on sampled patches (corners, edges, interior), (d) at
  full size the unperturbed case keeps the D4 symmetry bit for bit and the FP64
  totals of the FP32 state are conserved.
"""

import numpy as np
import pytest

import oracle
from paper_1401_0427_gb300 import inputs, lbm_sw

from gpu_helpers import FP32_ELEM_TOL, FP32_L1_TOL, FP64_TOL, rel_l1, rel_max, torch_stream

pytestmark = pytest.mark.gpu

P, W, O, I = lbm_sw.PERIODIC, lbm_sw.WALL, lbm_sw.OUTFLOW, lbm_sw.INFLOW


def _run_moments(nx, ny, W0, steps, *, dim=2, precision, bc, inflow=None, a):
    with lbm_sw.Simulation(nx, ny, dim=dim, precision=precision, bc=bc, inflow=inflow, a=a,
                           stream=torch_stream()) as sim:
        sim.set_state(*W0)
        sim.step(steps)
        return sim.moments()


# ------------------------------------------------------------------ 1D config
@pytest.fixture(scope="module")
def oracle_shock_tube():
    n, steps = 1000, 500
    h, q = inputs.dam_break_1d(n)
    p = oracle.params(n, a=0.15, bc=(oracle.WALL, oracle.WALL))
    return oracle.moments_1d(oracle.run_1d(oracle.equilibrium_1d(h, q, p), steps, p), p)


def test_shock_tube_1000_fp64(oracle_shock_tube):
    h, q = inputs.dam_break_1d(1000)
    gh, gq = _run_moments(1000, 1, (h, q), 500, dim=1, precision=lbm_sw.FP64, bc=(W, W), a=0.15)
    oh, oq = oracle_shock_tube
    assert rel_max(gh, oh) <= FP64_TOL and np.abs(gq - oq).max() <= FP64_TOL * np.abs(oh).max()


def test_shock_tube_1000_fp32(oracle_shock_tube):
    h, q = inputs.dam_break_1d(1000)
    gh, gq = _run_moments(1000, 1, (h, q), 500, dim=1, precision=lbm_sw.FP32, bc=(W, W), a=0.15)
    assert rel_l1(gh, oracle_shock_tube[0]) <= FP32_L1_TOL


# ------------------------------------------------------------------ 2D shock reflection
@pytest.fixture(scope="module")
def oracle_reflection_row():
    n, steps = 512, 2000
    uL = inputs.shock_speed_state(2.0, 1.0)
    inflow = [(2.0, 2.0 * uL, 0.0)] * 4
    p = oracle.params(n, 1, a=0.05, bc=(I, W, P, P), inflow=inflow)
    F = oracle.run_2d(oracle.equilibrium_2d(*inputs.planar_shock_2d(n, 1), p), steps, p)
    return oracle.moments_2d(F, p), inflow


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
def test_shock_reflection_512(oracle_reflection_row, precision):
    (oh, ohu, ohv), inflow = oracle_reflection_row
    n = 512
    gh, ghu, ghv = _run_moments(n, n, inputs.planar_shock_2d(n, n), 2000, precision=precision, bc=(I, W, P, P),
                                inflow=inflow, a=0.05)
    # y-invariance is exact on the GPU too
    assert np.array_equal(gh, np.broadcast_to(gh[:1], gh.shape))
    assert np.array_equal(ghu, np.broadcast_to(ghu[:1], ghu.shape))
    assert np.all(ghv == 0.0)
    if precision == lbm_sw.FP64:
        assert rel_max(gh[0], oh[0]) <= FP64_TOL
        assert np.abs(ghu[0] - ohu[0]).max() <= FP64_TOL * np.abs(oh).max()
    else:
        assert rel_l1(gh[0], oh[0]) <= FP32_L1_TOL
        assert np.abs(ghu[0] - ohu[0]).sum() / np.abs(oh[0]).sum() <= FP32_L1_TOL


# ------------------------------------------------------------------ 2D circular dam-break
@pytest.fixture(scope="module")
def oracle_dam_1024():
    n, steps = 1024, 250
    W0 = inputs.circular_dam_break_2d(n, seed=inputs.stream_seed(3, 1024))
    p = oracle.params(n, n, a=0.05)
    return W0, oracle.moments_2d(oracle.run_2d(oracle.equilibrium_2d(*W0, p), steps, p), p)


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
def test_dam_break_1024_full_run(oracle_dam_1024, precision):
    W0, (oh, ohu, ohv) = oracle_dam_1024
    gh, ghu, ghv = _run_moments(1024, 1024, W0, 250, precision=precision, bc=(P, P, P, P), a=0.05)
    if precision == lbm_sw.FP64:
        assert rel_max(gh, oh) <= FP64_TOL
        assert max(np.abs(ghu - ohu).max(), np.abs(ghv - ohv).max()) <= FP64_TOL * np.abs(oh).max()
    else:
        assert rel_l1(gh, oh) <= FP32_L1_TOL


def _patch_step(F, x0, y0, w, h):
    """Oracle's next post-collision state of the cells [y0, y0+h) x [x0, x0+w) from the
    post-collision state F (periodic domain): stream the patch with a one-cell halo
    (periodic wrap of the halo indices), then collide."""
    ny, nx = F.shape[1:]
    ys = np.arange(y0 - 1, y0 + h + 1) % ny
    xs = np.arange(x0 - 1, x0 + w + 1) % nx
    return _haloed_patch_step(F[:, ys][:, :, xs], w, h)


def _haloed_patch_step(sub, w, h):
    """The same from the patch with its one-cell halo, sub[13][h + 2][w + 2]."""
    sub = sub.astype(np.float64)
    p = oracle.params(w + 2, h + 2, a=0.05)
    streamed = oracle.stream_2d(np.ascontiguousarray(sub), p)  # halo ring is garbage, interior exact
    interior = np.ascontiguousarray(streamed[:, 1:-1, 1:-1])
    return oracle.collide_2d(interior, oracle.params(w, h, a=0.05))


@pytest.mark.slow
def test_dam_break_4096_whole_run_matches_oracle():
    """The circular dam-break workload as stated, in full: 4096 x 4096 periodic, 1000 steps
    from the seeded initial state.  The oracle runs the whole of it on every host core
    (1.7e10 FP64 cell updates, a few minutes, about 5 GB of host memory).  FP64 on the GPU:
    max |gpu - oracle| / max |oracle| <= 1e-12 for h, hu and hv.  FP32 on the GPU (the
    library's default kernel for this grid, 6 fused steps per launch): relative L1 of h
    <= 1e-5."""
    n, steps = 4096, 1000
    W0 = inputs.circular_dam_break_2d(n, seed=inputs.stream_seed(3))
    threads = oracle.set_threads(0)
    try:
        p = oracle.params(n, n, a=0.05)
        F = oracle.run_2d(oracle.equilibrium_2d(*W0, p), steps, p)
        oh, ohu, ohv = oracle.moments_2d(F, p)
        del F
    finally:
        oracle.set_threads(threads)
    gh, ghu, ghv = _run_moments(n, n, W0, steps, precision=lbm_sw.FP64, bc=(P, P, P, P), a=0.05)
    scale = np.abs(oh).max()
    assert rel_max(gh, oh) <= FP64_TOL
    assert max(np.abs(ghu - ohu).max(), np.abs(ghv - ohv).max()) <= FP64_TOL * scale
    fh, _, _ = _run_moments(n, n, W0, steps, precision=lbm_sw.FP32, bc=(P, P, P, P), a=0.05)
    assert rel_l1(fh, oh) <= FP32_L1_TOL


def test_dam_break_4096_sampled_step_parity():
    n = 4096
    W0 = inputs.circular_dam_break_2d(n, seed=inputs.stream_seed(3))
    with lbm_sw.Simulation(n, n, precision=lbm_sw.FP32, a=0.05, stream=torch_stream()) as sim:
        sim.set_state(*W0)
        sim.step(1000)
        Fk = sim.populations()
        sim.step(1)
        Fk1 = sim.populations()
    patches = [(0, 0), (n - 48, 0), (0, n - 48), (n - 48, n - 48), (2048 - 24, 2048 - 24), (1200, 1700),
               (3001, 17), (127, 2900)]
    for (x0, y0) in patches:
        want = _patch_step(Fk, x0, y0, 48, 48)
        got = Fk1[:, y0:y0 + 48, x0:x0 + 48].astype(np.float64)
        assert rel_max(got, want) <= FP32_ELEM_TOL, (x0, y0)


def test_dam_break_4096_d4_symmetry_and_conservation():
    n = 4096
    W0 = inputs.circular_dam_break_2d(n, seed=None)
    with lbm_sw.Simulation(n, n, precision=lbm_sw.FP32, a=0.05, stream=torch_stream()) as sim:
        sim.set_state(*W0)
        d0 = sim.diagnostics()
        sim.step(1000)
        d1 = sim.diagnostics()
        h, hu, hv = sim.moments()
    assert np.array_equal(h, h[::-1, :]) and np.array_equal(h, h[:, ::-1]) and np.array_equal(h, h.T)
    assert np.array_equal(hu, -hu[:, ::-1]) and np.array_equal(hu, hu[::-1, :]) and np.array_equal(hu, hv.T)
    assert h.max() < 2.0 + 1e-5 and not np.array_equal(h, W0[0])  # FP32 rounding of the untouched column
    assert abs(d1[0] - d0[0]) <= 1e-6 * d0[0]  # FP32 state, FP64 totals
    assert abs(d1[1]) <= 1e-6 * d0[0] and abs(d1[2]) <= 1e-6 * d0[0]


@pytest.mark.parametrize("bc", [(lbm_sw.PERIODIC,) * 4, (lbm_sw.WALL,) * 4], ids=["periodic", "walls"])
def test_dam_break_fp64_d4_symmetry(bc):
    """FP64 (the folded BGK form): mirror-image cells see mirror-image operations, so the
    circular dam-break keeps the symmetries of the square bit for bit."""
    n = 256
    W0 = inputs.circular_dam_break_2d(n, seed=None)
    with lbm_sw.Simulation(n, n, precision=lbm_sw.FP64, a=0.05, bc=bc, stream=torch_stream()) as sim:
        sim.set_state(*W0)
        sim.step(300)
        h, hu, hv = sim.moments()
    assert np.array_equal(h, h[::-1, :]) and np.array_equal(h, h[:, ::-1]) and np.array_equal(h, h.T)
    assert np.array_equal(hu, -hu[:, ::-1]) and np.array_equal(hu, hu[::-1, :]) and np.array_equal(hu, hv.T)
    assert not np.array_equal(h, W0[0])


def test_grid_past_32_bit_indices():
    """16384 x 12288 cells in FP32: each population buffer holds 2.6e9 elements, past 32-bit
    indexing.  The temporal kernel (6 steps per launch) equals 6 single steps bit for bit,
    and one more step on patches at the far end of the buffers (the last rows and columns)
    matches the oracle.  The state is a seeded random 1024 x 1536 tile repeated."""
    import torch

    nx, ny, tw, th = 16384, 12288, 1024, 1536
    tile = inputs.random_states(tw * th, seed=inputs.stream_seed(7), h=(0.8, 1.4), speed=0.25)
    W0 = [np.tile(w.reshape(th, tw), (ny // th, nx // tw)) for w in tile]
    out = []
    for kernel in (lbm_sw.KERNEL_TEMPORAL, lbm_sw.KERNEL_VEC):
        with lbm_sw.Simulation(nx, ny, precision=lbm_sw.FP32, a=0.05, kernel=kernel, stream=torch_stream()) as sim:
            assert sim.info().steps_per_launch == (6 if kernel == lbm_sw.KERNEL_TEMPORAL else 1)
            sim.set_state(*W0)
            sim.step(6)
            F = torch.empty((13, ny, nx), dtype=torch.float32, device="cuda")
            sim.populations_into(F)
            out.append(F)
            if kernel == lbm_sw.KERNEL_VEC:
                sim.step(1)
                F1 = torch.empty_like(F)
                sim.populations_into(F1)
    assert torch.equal(out[0], out[1])
    F = out[1]
    for x0, y0 in [(nx - 40, ny - 40), (0, ny - 40), (nx - 40, 0), (8190, ny - 40)]:
        ys = torch.arange(y0 - 1, y0 + 41, device="cuda") % ny
        xs = torch.arange(x0 - 1, x0 + 41, device="cuda") % nx
        sub = F[:, ys][:, :, xs].cpu().numpy()
        want = _haloed_patch_step(sub, 40, 40)
        got = F1[:, y0:y0 + 40, x0:x0 + 40].cpu().numpy().astype(np.float64)
        assert rel_max(got, want) <= FP32_ELEM_TOL, (x0, y0)
