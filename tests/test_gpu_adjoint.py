"""Discrete adjoint (lbm_sw_tape_* / lbm_sw_adjoint) against complex-step derivatives and
central finite differences of the FP64 oracle.

For L = 1/2 sum (h_T - h_obs)^2 after T steps from f = f^eq(W0), the directional
derivative dL/dW0 . delta from the GPU adjoint must equal Im L(W0 + i eps delta) / eps
computed by the oracle in complex arithmetic (the scheme is analytic in W0; eps = 1e-30),
on random directions and single cells, for periodic and mixed (wall / outflow / inflow)
boundaries, in the h and hu components.  FP64 to 1e-9; FP32 (FP32 states and adjoint,
FP64 checkpoints) to 2e-3 relative (the adjoint accumulates FP32 rounding over T steps).
"""

import numpy as np
import pytest

import oracle
from paper_1401_0427_gb300 import inputs, lbm_sw

from gpu_helpers import torch_stream

pytestmark = pytest.mark.gpu

P, W, O, I = lbm_sw.PERIODIC, lbm_sw.WALL, lbm_sw.OUTFLOW, lbm_sw.INFLOW
INFLOW = [(1.1, 0.1, 0.0), (1.0, 0.0, 0.0), (1.05, 0.0, 0.08), (1.0, 0.0, 0.0)]


def _workload(n, seed_true=5, seed_guess=6):
    h_true = inputs.gaussian_bumps_2d(n, seed=inputs.stream_seed(5, seed_true))[0]
    h_guess = 1.0 + 0.5 * (h_true - 1.0)
    return h_true, h_guess


def _oracle_hT(W0, steps, p):
    F = oracle.run_2d(oracle.equilibrium_2d(*W0, p), steps, p)
    return oracle.moments_2d(F, p)[0]


def _oracle_directional(W0, dW, steps, p, h_obs):
    """Im L(W0 + i eps dW) / eps with the oracle in complex arithmetic."""
    eps = 1e-30
    Wc = [W0[k] + 1j * eps * dW[k] for k in range(3)]
    F = oracle.run_2d_cplx(oracle.equilibrium_2d_cplx(*Wc, p), steps, p)
    hT = F[0] + ((F[1] + F[3]) + (F[2] + F[4]))
    L = 0.5 * ((hT - h_obs) ** 2).sum()
    return L.imag / eps


def _gpu_gradient(W0, steps, h_obs, *, precision, bc=(P,) * 4, interval=0, kernel=lbm_sw.KERNEL_AUTO):
    ny, nx = W0[0].shape
    with lbm_sw.Simulation(nx, ny, precision=precision, bc=bc, inflow=INFLOW, stream=torch_stream(),
                           kernel=kernel) as sim:
        sim.set_state(*W0)
        with lbm_sw.Tape(sim, steps, interval) as tape:
            tape.record()
            hT = sim.moments()[0]
            grads = tape.adjoint(hT - h_obs, want_momentum=True)
            info = tape.info()
    return grads, hT, info


def _directions(n, count, seed):
    out = [inputs.uniform(seed + k, n * n, -1, 1).reshape(n, n) for k in range(count)]
    rng = np.random.default_rng(seed)
    for _ in range(count):
        e = np.zeros((n, n))
        e[rng.integers(n), rng.integers(n)] = 1.0
        out.append(e)
    return out


def test_fp64_gradient_matches_complex_step_periodic_64():
    n, steps = 64, 200
    h_true, h_guess = _workload(n)
    z = np.zeros((n, n))
    p = oracle.params(n, n, a=0.05)
    h_obs = _oracle_hT((h_true, z, z), steps, p)
    (gh, gu, gv), hT, info = _gpu_gradient((h_guess, z, z), steps, h_obs, precision=lbm_sw.FP64)
    assert info.interval == 15 and info.checkpoints == 14
    for d in _directions(n, 6, 300):
        want = _oracle_directional((h_guess, z, z), (d, z, z), steps, p, h_obs)
        got = float((gh * d).sum())
        assert abs(got - want) <= 1e-9 * max(abs(want), 1e-3), (got, want)


def _oracle_loss(W0, steps, p, h_obs):
    hT = _oracle_hT(W0, steps, p)
    return 0.5 * float(((hT - h_obs) ** 2).sum())


def test_fp64_gradient_matches_central_differences_of_the_oracle_64():
    """The same gradient against central finite differences of the FP64 oracle,
    (L(W0 + eps d) - L(W0 - eps d)) / (2 eps) with eps = 1e-6, along random and single-cell
    directions of h and random directions of hu and hv.  The difference quotient is accurate
    to about 1e-8 here: its truncation error is of order eps^2 times the third derivative of
    L (~ 1e-11), and the rounding of the two losses (L ~ 10, relative rounding ~ 1e-15 after
    200 steps) contributes ~ 1e-14 / 2e-6 ~ 1e-8; the bar is 1e-6 relative."""
    n, steps, eps = 64, 200, 1e-6
    h_true, h_guess = _workload(n)
    z = np.zeros((n, n))
    p = oracle.params(n, n, a=0.05)
    h_obs = _oracle_hT((h_true, z, z), steps, p)
    W0 = (h_guess, z, z)
    grads, _, _ = _gpu_gradient(W0, steps, h_obs, precision=lbm_sw.FP64)
    cases = [(0, d) for d in _directions(n, 3, 700)]
    cases += [(comp, inputs.uniform(710 + comp, n * n, -1, 1).reshape(n, n)) for comp in (1, 2)]
    for comp, d in cases:
        plus = [w.copy() for w in W0]
        minus = [w.copy() for w in W0]
        plus[comp] += eps * d
        minus[comp] -= eps * d
        want = (_oracle_loss(plus, steps, p, h_obs) - _oracle_loss(minus, steps, p, h_obs)) / (2 * eps)
        got = float((grads[comp] * d).sum())
        assert abs(got - want) <= 1e-6 * max(abs(want), 1e-3), (comp, got, want)


@pytest.mark.parametrize("bc", [(W, O, I, W), (I, W, P, P), (O, O, W, W)], ids=["WOIW", "IWPP", "OOWW"])
def test_fp64_gradient_matches_complex_step_mixed_boundaries(bc):
    nx, ny, steps = 24, 16, 30
    W0 = [x.reshape(ny, nx) for x in inputs.random_states(nx * ny, seed=410, h=(0.8, 1.4), speed=0.25)]
    W1 = [x.reshape(ny, nx) for x in inputs.random_states(nx * ny, seed=411, h=(0.8, 1.4), speed=0.25)]
    p = oracle.params(nx, ny, a=0.05, bc=bc, inflow=INFLOW)
    h_obs = _oracle_hT(W1, steps, p)
    grads, _, _ = _gpu_gradient(W0, steps, h_obs, precision=lbm_sw.FP64, bc=bc)
    rng = np.random.default_rng(412)
    for comp in range(3):
        for k in range(3):
            d = rng.uniform(-1, 1, (ny, nx))
            dW = [np.zeros((ny, nx)) for _ in range(3)]
            dW[comp] = d
            want = _oracle_directional(W0, dW, steps, p, h_obs)
            got = float((grads[comp] * d).sum())
            assert abs(got - want) <= 1e-9 * max(abs(want), 1e-3), (comp, got, want)


def test_checkpoint_interval_does_not_change_the_gradient():
    """The segment logic must not change the result: only rounding may differ (at a
    checkpoint the moments are summed from the stored post-collision state, inside a
    replayed step from the pre-collision one; the collision conserves them exactly in
    exact arithmetic only)."""
    nx, ny, steps = 40, 24, 37
    W0 = [x.reshape(ny, nx) for x in inputs.random_states(nx * ny, seed=420, h=(0.8, 1.4), speed=0.25)]
    h_obs = np.ones((ny, nx))
    ref = None
    for interval in (1, 4, 7, 0, 37):
        for prec in (lbm_sw.FP64,):
            g, _, info = _gpu_gradient(W0, steps, h_obs, precision=prec, bc=(W, O, P, P), interval=interval)
            if ref is None:
                ref = g
            else:
                for a, b in zip(g, ref):
                    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), interval


def test_fp32_gradient_matches_complex_step_64():
    n, steps = 64, 200
    h_true, h_guess = _workload(n)
    z = np.zeros((n, n))
    p = oracle.params(n, n, a=0.05)
    h_obs = _oracle_hT((h_true, z, z), steps, p)
    (gh, _, _), _, _ = _gpu_gradient((h_guess, z, z), steps, h_obs, precision=lbm_sw.FP32)
    for d in _directions(n, 4, 500)[:6]:
        want = _oracle_directional((h_guess, z, z), (d, z, z), steps, p, h_obs)
        got = float((gh * d).sum())
        assert abs(got - want) <= 2e-3 * max(abs(want), 1e-3), (got, want)


def test_inverse_problem_workload_1024():
    """1024 x 1024 periodic, 8 Gaussian bumps, T = 200, FP32 with FP64 checkpoints: the FP32
    gradient against the FP64 one (relative L2) and one direction against the oracle."""
    n, steps = 1024, 200
    h_true, h_guess = _workload(n)
    z = np.zeros((n, n))
    p = oracle.params(n, n, a=0.05)
    h_obs = _oracle_hT((h_true, z, z), steps, p)
    (g64, _, _), _, _ = _gpu_gradient((h_guess, z, z), steps, h_obs, precision=lbm_sw.FP64)
    (g32, _, _), _, info = _gpu_gradient((h_guess, z, z), steps, h_obs, precision=lbm_sw.FP32)
    # the FP32 handle fuses 6 steps per launch forward and 4 in the replay: the default
    # interval ceil(sqrt(200)) = 15 is rounded up to 24, so 9 checkpoints
    assert info.interval == 24 and info.checkpoints == 9
    assert info.checkpoint_bytes == 9 * 13 * 1024 * 1024 * 8
    assert np.linalg.norm(g32 - g64) <= 2e-3 * np.linalg.norm(g64)
    d = inputs.uniform(77, n * n, -1, 1).reshape(n, n)
    want = _oracle_directional((h_guess, z, z), (d, z, z), steps, p, h_obs)
    assert abs(float((g64 * d).sum()) - want) <= 1e-9 * abs(want)
    # one interval of T steps: the recorded run keeps the moments of every step and the
    # backward pass replays nothing; the adjoint launches split the steps differently, so the
    # gradient agrees to FP32 rounding
    (gT, _, _), _, infoT = _gpu_gradient((h_guess, z, z), steps, h_obs, precision=lbm_sw.FP32, interval=steps)
    assert infoT.interval == steps and infoT.checkpoints == 1
    assert np.abs(gT - g32).max() <= 1e-5 * np.abs(g32).max()


def test_autograd_function_and_recovery():
    import torch

    from paper_1401_0427_gb300 import adjoint

    n, steps = 128, 100
    h_true, h_guess = _workload(n)
    dev = torch.device("cuda")
    with lbm_sw.Simulation(n, n, precision=lbm_sw.FP64, stream=torch_stream()) as sim:
        ht = torch.tensor(h_true, device=dev)
        h_obs = adjoint.run(ht, sim, steps).detach()
        h0 = torch.tensor(h_guess, device=dev, requires_grad=True)
        loss = 0.5 * ((adjoint.run(h0, sim, steps) - h_obs) ** 2).sum()
        loss.backward()
        g_auto = h0.grad.cpu().numpy()
        (g_tape, _, _), _, _ = _gpu_gradient((h_guess, np.zeros((n, n)), np.zeros((n, n))), steps,
                                             h_obs.cpu().numpy(), precision=lbm_sw.FP64)
        assert np.allclose(g_auto, g_tape, rtol=0, atol=1e-12 * np.abs(g_tape).max())
        h_fit, losses = adjoint.recover_initial_depth(h_obs, sim, steps, torch.tensor(h_guess, device=dev),
                                                      iterations=15)
    assert losses[-1] < 0.05 * losses[0]
    err0 = np.abs(h_guess - h_true).mean()
    err1 = np.abs(h_fit.cpu().numpy() - h_true).mean()
    assert err1 < 0.5 * err0


def test_autograd_backward_twice_with_retain_graph():
    """The tape lives as long as the autograd graph: a second backward (retain_graph=True)
    replays the same checkpoints and doubles the accumulated gradient; the forward pass leaves
    the caller's Simulation at step T."""
    import torch

    from paper_1401_0427_gb300 import adjoint

    n, steps = 64, 40
    h_true, h_guess = _workload(n)
    dev = torch.device("cuda")
    with lbm_sw.Simulation(n, n, precision=lbm_sw.FP64, stream=torch_stream()) as sim:
        h_obs = torch.tensor(h_true, device=dev)
        h0 = torch.tensor(h_guess, device=dev, requires_grad=True)
        hT = adjoint.run(h0, sim, steps)
        assert sim.info().steps_done == steps
        assert np.array_equal(sim.moments()[0], hT.detach().cpu().numpy())
        loss = 0.5 * ((hT - h_obs) ** 2).sum()
        loss.backward(retain_graph=True)
        g1 = h0.grad.clone()
        loss.backward()
        assert torch.equal(h0.grad, 2 * g1)


def _gradient_with_kernel(W0, steps, h_obs, precision, bc, kernel):
    ny, nx = W0[0].shape
    with lbm_sw.Simulation(nx, ny, precision=precision, bc=bc, inflow=INFLOW, kernel=kernel,
                           stream=torch_stream()) as sim:
        sim.set_state(*W0)
        with lbm_sw.Tape(sim, steps) as tape:
            tape.record()
            return tape.adjoint(sim.moments()[0] - h_obs, want_momentum=True)


@pytest.mark.parametrize("precision", [lbm_sw.FP64, lbm_sw.FP32])
@pytest.mark.parametrize("bc", [(P, P, P, P), (W, O, I, W), (O, I, W, O), (W, W, W, W), (I, W, P, P)],
                         ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 2), (1, 5), (7, 5), (64, 3), (130, 9), (257, 33)])
def test_vector_adjoint_equals_scalar_adjoint(nx, ny, bc, precision):
    """The vectorised adjoint step (warp shuffles, vector loads, warp-uniform boundary
    branches) against the one-thread-per-cell adjoint step on ragged grids."""
    steps = 9
    W0 = [x.reshape(ny, nx) for x in inputs.random_states(nx * ny, seed=430 + nx, h=(0.8, 1.4), speed=0.25)]
    h_obs = np.ones((ny, nx))
    a = _gradient_with_kernel(W0, steps, h_obs, precision, bc, lbm_sw.KERNEL_SIMPLE)
    b = _gradient_with_kernel(W0, steps, h_obs, precision, bc, lbm_sw.KERNEL_VEC)
    tol = 1e-13 if precision == lbm_sw.FP64 else 1e-5
    for ga, gb in zip(a, b):
        assert np.abs(ga - gb).max() <= tol * max(np.abs(ga).max(), 1e-30)


def test_fused_launches_give_the_same_fp32_gradient():
    """1024 x 1024 periodic FP32: the default handle fuses 6 steps per launch in the forward
    run and in the segment replays (whose kernel also stores every level's moments), and 4 in
    the adjoint steps (a reverse wavefront of the same shape); a handle held to one step per
    launch gives the same gradient, with intervals of 16 (fused adjoint launches only) and 15
    (fused launches and single steps).  The forward run and the replays are bit-identical; the
    two adjoint kernels evaluate the same plain-arithmetic expressions, whose contraction into
    fused multiply-adds the compiler may choose per kernel, so they agree to FP32 rounding.
    With walls, outflow and inflow the forward run and the replays are fused, the adjoint
    steps single."""
    n, steps = 1024, 48
    h_true, h_guess = _workload(n)
    z = np.zeros((n, n))
    p = oracle.params(n, n, a=0.05)
    h_obs = _oracle_hT((h_true, z, z), steps, p)
    for interval in (16, 15):
        fused, hT_f, _ = _gpu_gradient((h_guess, z, z), steps, h_obs, precision=lbm_sw.FP32, interval=interval)
        single, hT_s, _ = _gpu_gradient((h_guess, z, z), steps, h_obs, precision=lbm_sw.FP32, interval=interval,
                                        kernel=lbm_sw.KERNEL_VEC)
        assert np.array_equal(hT_f, hT_s)
        for a, b in zip(fused, single):
            assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max(), interval
    # walls, outflow and inflow: fused forward run and replays, single adjoint steps in both
    bc = (W, O, I, W)
    fused, hT_f, _ = _gpu_gradient((h_guess, z, z), steps, h_obs, precision=lbm_sw.FP32, bc=bc, interval=15)
    single, hT_s, _ = _gpu_gradient((h_guess, z, z), steps, h_obs, precision=lbm_sw.FP32, bc=bc, interval=15,
                                    kernel=lbm_sw.KERNEL_VEC)
    assert np.array_equal(hT_f, hT_s)
    for a, b in zip(fused, single):
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()


@pytest.mark.parametrize("nx,ny", [(2, 3), (7, 5), (10, 7), (246, 9), (250, 33), (300, 40), (501, 20)])
@pytest.mark.parametrize("k", [2, 4, 6, 8])
def test_fused_adjoint_on_ragged_grids(nx, ny, k):
    """FP32 periodic handles held to temporal blocking with K = 2 .. 8 (adjoint launches of
    min(K, 4) reverse steps: two columns per thread for even widths, one otherwise) against
    one step per launch, on grids around the strip widths: the forward run is bit-identical,
    the gradient equal to FP32 rounding."""
    steps = 24
    W0 = [x.reshape(ny, nx) for x in inputs.random_states(nx * ny, seed=470 + nx + ny, h=(0.8, 1.4), speed=0.25)]
    h_obs = np.ones((ny, nx))
    out = []
    for kernel in (lbm_sw.KERNEL_TEMPORAL, lbm_sw.KERNEL_VEC):
        with lbm_sw.Simulation(nx, ny, precision=lbm_sw.FP32, kernel=kernel, temporal_steps=k,
                               stream=torch_stream()) as sim:
            sim.set_state(*W0)
            with lbm_sw.Tape(sim, steps) as tape:
                tape.record()
                hT = sim.moments()[0]
                out.append((hT, tape.adjoint(hT - h_obs, want_momentum=True)))
    (h_a, g_a), (h_b, g_b) = out
    assert np.array_equal(h_a, h_b)
    for a, b in zip(g_a, g_b):
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()


@pytest.mark.parametrize("bc", [(W, W, W, W), (W, O, I, W), (I, W, P, P), (O, I, W, O), (P, P, W, O), (O, O, O, O)],
                         ids=lambda b: "".join("PWOI"[k] for k in b))
@pytest.mark.parametrize("nx,ny", [(2, 3), (10, 1), (10, 2), (7, 5), (246, 9), (250, 33)])
@pytest.mark.parametrize("k", [2, 4])
def test_fused_adjoint_with_boundaries(nx, ny, bc, k):
    """The reverse wavefront with the transposed rules of walls, inflow and outflow (two
    columns per thread, even widths; odd widths take single adjoint steps) against one adjoint
    step per launch, on grids one or two rows high and one pair wide among others.  The bound
    is FP32 rounding of the gradient's scale (its largest component): in one row between two
    walls dL/dhv is orders of magnitude below dL/dh and carries the same absolute rounding."""
    steps = 24
    W0 = [x.reshape(ny, nx) for x in inputs.random_states(nx * ny, seed=520 + nx + ny, h=(0.8, 1.4), speed=0.25)]
    h_obs = np.ones((ny, nx))
    out = []
    for kernel in (lbm_sw.KERNEL_TEMPORAL, lbm_sw.KERNEL_VEC):
        with lbm_sw.Simulation(nx, ny, precision=lbm_sw.FP32, kernel=kernel, temporal_steps=k, bc=bc, inflow=INFLOW,
                               stream=torch_stream()) as sim:
            sim.set_state(*W0)
            with lbm_sw.Tape(sim, steps) as tape:
                tape.record()
                hT = sim.moments()[0]
                out.append((hT, tape.adjoint(hT - h_obs, want_momentum=True)))
    (h_a, g_a), (h_b, g_b) = out
    assert np.array_equal(h_a, h_b)
    scale = max(np.abs(b).max() for b in g_b)
    for a, b in zip(g_a, g_b):
        assert np.abs(a - b).max() <= 1e-5 * scale
