"""Pins of whole oracle runs against the mathematics of the shallow-water equations.

* 1D dam-break (section 2 shock tube; the paper's Figure 1 compares with the exact
  solution): the D1Q3Q2 scheme converges in L1 toward Stoker's solution as the mesh
  is refined at fixed time, for the benchmark case (h_r = 1) and the paper's case
  (rho_r / rho_0 = 0.5), with the paper's lambda/c0 = 8, a = 0.15, s = 1.8.
* The D2Q5Q4Q4 scheme on a y-invariant dam-break converges toward the same solution.
* A planar shock reflected by a wall leaves the Rankine-Hugoniot depth behind it.
* Symmetries: y-invariance and the D4 symmetry of a centred circular dam-break are
  kept bit for bit (moments are summed in mirror-symmetric pairs).
* Conservation: total mass on periodic and walled domains, total momentum on
  periodic domains, to round-off.
* Complex-step derivatives of a run agree with central differences.
* The shock-reflection states printed in section 4 satisfy the Rankine-Hugoniot
  conditions of the shallow-water system with g = 1.
"""

import math
import os

import numpy as np
import pytest

import oracle
from oracle import INFLOW, OUTFLOW, PERIODIC, WALL
from paper_1401_0427_gb300 import inputs

from exact import oblique_jump_residual, stoker, stoker_profile, wall_reflection

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _run_dam_1d(n, h_right, steps, a=0.15, lam=8.0, s=1.8):
    p = oracle.params(n, a=a, lam=lam, s=s, bc=(WALL, WALL))
    h, q = inputs.dam_break_1d(n, 2.0, h_right)
    F = oracle.run_1d(oracle.equilibrium_1d(h, q, p), steps, p)
    return oracle.moments_1d(F, p)


def test_stoker_constants():
    hs, us, shock, head, tail = stoker(2.0, 1.0)
    assert abs(hs - 1.453840892374573) < 1e-13 and abs(us - 0.416920630975483) < 1e-13
    assert abs(shock - 1.335569959364740) < 1e-12 and abs(tail + 0.788832615909871) < 1e-12
    hs, us, *_ = stoker(2.0, 0.5)
    assert abs(hs - 1.103493853837107) < 1e-12 and abs(us - 0.727480810499101) < 1e-12


@pytest.mark.parametrize("h_right", [1.0, 0.5])
def test_1d_dam_break_converges_to_stoker(h_right):
    """T = 500 dt at N = 1000 with lambda = 8 (t = 0.0625): waves stay off the walls."""
    errs = []
    sizes = [250, 500, 1000, 2000, 4000]
    for n in sizes:
        steps = n // 2
        t = steps / (n * 8.0)
        h, q = _run_dam_1d(n, h_right, steps)
        he, ue = stoker_profile(inputs.cell_centres(n), t, 2.0, h_right)
        errs.append((np.abs(h - he).mean(), np.abs(q / h - ue).mean()))
    errs = np.array(errs)
    assert np.all(np.diff(errs[:, 0]) < 0) and np.all(np.diff(errs[:, 1]) < 0)
    order = np.log2(errs[:-1, 0] / errs[1:, 0])
    assert order.min() > 0.5, order
    assert errs[-1, 0] < 2e-3


def test_paper_shock_tube_80_points_reaches_the_middle_state():
    """The paper's own run: 80 points, rho_l/rho_0 = 2, rho_r/rho_0 = 0.5, run to t = 1/4
    (160 steps) when the exact middle state spans 0.42 < x < 0.83."""
    n = 80
    h, q = _run_dam_1d(n, 0.5, 160)
    assert np.all(np.isfinite(h)) and h.min() > 0.49 and h.max() < 2.01
    hs, us, *_ = stoker(2.0, 0.5)
    x = inputs.cell_centres(n)
    mid = (x > 0.55) & (x < 0.72)
    assert np.all(np.abs(h[mid] - hs) < 0.05 * hs)
    assert np.all(np.abs(q[mid] / h[mid] - us) < 0.05 * us)


def test_2d_y_invariant_dam_break_converges_to_stoker():
    errs = []
    for n in [200, 400, 800, 1600]:
        steps = n // 2
        t = steps / (n * 8.0)
        p = oracle.params(n, 1, a=0.05, bc=(WALL, WALL, PERIODIC, PERIODIC))
        h0, q0 = inputs.dam_break_1d(n)
        F = oracle.run_2d(oracle.equilibrium_2d(h0, q0, 0 * q0, p), steps, p)
        h, _, _ = oracle.moments_2d(F, p)
        he, _ = stoker_profile(inputs.cell_centres(n), t, 2.0, 1.0)
        errs.append(np.abs(h[0] - he).mean())
    assert np.all(np.diff(errs) < 0), errs
    assert np.log2(errs[-2] / errs[-1]) > 0.5


def test_shock_reflection_plateau_matches_rankine_hugoniot():
    """The benchmark shock-reflection layout at 512 cells across (y-invariant, so one row
    stands for the whole grid): inflow of the left state on x-, wall on x+."""
    n, steps = 512, 2000
    uL = inputs.shock_speed_state(2.0, 1.0)
    p = oracle.params(n, 1, a=0.05, bc=(INFLOW, WALL, PERIODIC, PERIODIC), inflow=[(2.0, 2.0 * uL, 0.0)] * 4)
    h0, hu0, hv0 = inputs.planar_shock_2d(n, 1)
    F = oracle.run_2d(oracle.equilibrium_2d(h0, hu0, hv0, p), steps, p)
    h, hu, _ = oracle.moments_2d(F, p)
    h2, speed = wall_reflection(2.0, uL)
    assert abs(h2 - 3.372281323269014) < 1e-12
    t = steps / (n * 8.0)
    t_hit = 0.5 / math.sqrt(3.0)
    x_shock = 1.0 + speed * (t - t_hit)
    x = inputs.cell_centres(n)
    plateau = (x > x_shock + 0.04) & (x < 0.98)
    assert plateau.sum() > 60
    assert np.all(np.abs(h[0, plateau] - h2) < 0.01 * h2)
    assert np.all(np.abs(hu[0, plateau]) < 0.02)
    # the reflected shock sits where Rankine-Hugoniot puts it (numerical width ~ a few cells)
    mid = x[np.argmin(np.abs(h[0] - (h2 + 2.0) / 2.0) + 10.0 * (x < 0.6))]
    assert abs(mid - x_shock) < 0.02


def test_y_invariance_is_exact():
    nx, ny, steps = 64, 6, 120
    uL = inputs.shock_speed_state(2.0, 1.0)
    p = oracle.params(nx, ny, a=0.05, bc=(INFLOW, WALL, PERIODIC, PERIODIC), inflow=[(2.0, 2.0 * uL, 0.0)] * 4)
    F = oracle.run_2d(oracle.equilibrium_2d(*inputs.planar_shock_2d(nx, ny), p), steps, p)
    assert np.array_equal(F, np.broadcast_to(F[:, :1, :], F.shape))


def _d4_images(F):
    """The 8 images of a 2D population field under the symmetries of the square, with
    populations permuted and momentum families re-signed to match."""
    f, gx, gy = F[0:5], F[5:9], F[9:13]

    def mirror_x(f, gx, gy):  # x -> -x: v1 <-> v3, gx -> -gx
        perm = [0, 3, 2, 1, 4]
        return f[perm][:, :, ::-1], -gx[[2, 1, 0, 3]][:, :, ::-1], gy[[2, 1, 0, 3]][:, :, ::-1]

    def transpose(f, gx, gy):  # x <-> y: v1 <-> v2, v3 <-> v4, gx <-> gy
        perm = [0, 2, 1, 4, 3]
        p4 = [1, 0, 3, 2]
        return (f[perm].transpose(0, 2, 1), gy[p4].transpose(0, 2, 1), gx[p4].transpose(0, 2, 1))

    out = []
    cur = (f, gx, gy)
    for _ in range(2):
        for _ in range(2):
            for _ in range(2):
                out.append(np.concatenate(cur))
                cur = mirror_x(*cur)
            cur = transpose(*cur)
        cur = mirror_x(*transpose(*mirror_x(*transpose(*cur))))
    return out


@pytest.mark.parametrize("bc", [PERIODIC, WALL, OUTFLOW])
def test_circular_dam_break_keeps_d4_symmetry_bitwise(bc):
    n, steps = 48, 60
    p = oracle.params(n, n, a=0.05, bc=(bc,) * 4)
    h, hu, hv = inputs.circular_dam_break_2d(n, seed=None, radius=0.2)
    F = oracle.run_2d(oracle.equilibrium_2d(h, hu, hv, p), steps, p)
    images = _d4_images(F)
    assert len(images) == 8
    for im in images:
        assert np.array_equal(im, F)
    hh, _, _ = oracle.moments_2d(F, p)
    assert hh.max() < 2.0 and hh.min() > 0.9 and not np.array_equal(hh, h)


@pytest.mark.parametrize("bc", [PERIODIC, WALL])
def test_mass_and_momentum_conservation(bc):
    n, steps = 40, 300
    p = oracle.params(n, n, a=0.05, bc=(bc,) * 4)
    h, hu, hv = inputs.circular_dam_break_2d(n, seed=inputs.stream_seed(3), perturbation=1e-3)
    hu = hu + 0.05 * inputs.uniform(7, n * n, -1, 1).reshape(n, n)
    F0 = oracle.equilibrium_2d(h, hu, hv, p)
    F = oracle.run_2d(F0, steps, p)
    m0 = [x.sum() for x in oracle.moments_2d(F0, p)]
    m1 = [x.sum() for x in oracle.moments_2d(F, p)]
    assert abs(m1[0] - m0[0]) <= 1e-13 * m0[0]
    if bc == PERIODIC:
        assert abs(m1[1] - m0[1]) <= 1e-13 * m0[0] and abs(m1[2] - m0[2]) <= 1e-13 * m0[0]


def test_1d_mass_conservation_walls():
    n = 500
    p = oracle.params(n, a=0.15, bc=(WALL, WALL))
    h, q = inputs.dam_break_1d(n)
    F0 = oracle.equilibrium_1d(h, q, p)
    F = oracle.run_1d(F0, 2000, p)  # long enough for many wall reflections
    assert abs(oracle.moments_1d(F, p)[0].sum() - h.sum()) <= 1e-13 * h.sum()


@pytest.mark.parametrize("perturb", [0, 1, 2], ids=["h", "hu", "hv"])
def test_complex_step_matches_central_differences(perturb):
    """The derivative of a 2D run along a perturbation of h, hu or hv: complex step equals
    central differences, and the real part of the complex run is the real run."""
    nx, ny, steps = 8, 6, 12
    p = oracle.params(nx, ny, a=0.05, bc=(WALL, PERIODIC, OUTFLOW, INFLOW), inflow=[(1.2, 0.1, 0.05)] * 4)
    W0 = inputs.random_states(nx * ny, seed=51, h=(0.8, 1.6), speed=0.3)
    d = inputs.uniform(52, nx * ny, -1, 1)
    probe = inputs.uniform(53, 13 * nx * ny, -1, 1).reshape(13, ny, nx)

    def W(t):
        return [w + t * d if k == perturb else w for k, w in enumerate(W0)]

    def J(t):
        return float((oracle.run_2d(oracle.equilibrium_2d(*W(t), p), steps, p) * probe).sum())

    eps = 1e-6
    fd = (J(eps) - J(-eps)) / (2 * eps)
    Fc = oracle.run_2d_cplx(oracle.equilibrium_2d_cplx(*W(1e-30j), p), steps, p)
    cs = float((Fc.imag * probe).sum()) / 1e-30
    assert abs(cs - fd) <= 1e-7 * max(1.0, abs(cs))
    # the complex run's real part is the real run
    assert np.allclose(Fc.real, oracle.run_2d(oracle.equilibrium_2d(*W(0.0), p), steps, p), rtol=0, atol=1e-15)


@pytest.mark.parametrize("perturb", ["h", "q"])
def test_complex_step_matches_central_differences_1d(perturb):
    """The 1D complex-step entry points: the derivative of a 1D run (walls on one side,
    inflow on the other) along a perturbation of h or q equals central differences, and the
    real part of the complex run is the real run."""
    n, steps = 24, 15
    p = oracle.params(n, a=0.15, bc=(WALL, INFLOW), inflow=[None, (1.1, -0.05, 0.0), None, None])
    h, q, _ = inputs.random_states(n, seed=61, h=(0.8, 1.6), speed=0.3)
    d = inputs.uniform(62, n, -1, 1)
    probe = inputs.uniform(63, 5 * n, -1, 1).reshape(5, n)

    def W(t):
        return (h + t * d, q) if perturb == "h" else (h, q + t * d)

    def J(t):
        return float((oracle.run_1d(oracle.equilibrium_1d(*W(t), p), steps, p) * probe).sum())

    eps = 1e-6
    fd = (J(eps) - J(-eps)) / (2 * eps)
    Fc = oracle.run_1d_cplx(oracle.equilibrium_1d_cplx(*W(1e-30j), p), steps, p)
    cs = float((Fc.imag * probe).sum()) / 1e-30
    assert abs(cs - fd) <= 1e-7 * max(1.0, abs(cs))
    assert np.allclose(Fc.real, oracle.run_1d(oracle.equilibrium_1d(*W(0.0), p), steps, p), rtol=0, atol=1e-15)


def _golden_states():
    rows = {}
    with open(os.path.join(GOLDEN, "e2_shock_reflection_states.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, *vals = line.split()
                rows[name] = tuple(float(v) for v in vals)
    return rows


def test_printed_shock_reflection_states_satisfy_rankine_hugoniot_with_g_1():
    st = _golden_states()
    r = oblique_jump_residual(st["left"], st["top"], -math.pi / 4)
    assert np.abs(r).max() < 1e-13
    # the reflected shock: find the line angle that makes the tangential velocity continuous,
    # then check the two flux conditions there
    t, rr = st["top"], st["right"]
    du = np.array([rr[1] - t[1], rr[2] - t[2]])  # velocity jump is normal to the shock
    angle = math.atan2(du[0], -du[1])
    res = oblique_jump_residual(t, rr, angle)
    assert np.abs(res).max() < 1e-12
    assert abs(math.tan(angle) - 1.25) < 1e-9 or abs(math.tan(angle + math.pi) - 1.25) < 1e-9
