"""Pins of the oracle's streaming and boundary rules.

With s = 0 the collision is the identity, so a run is pure streaming
f_j(x + v_j dt) = f_j*(x) (lambda = dx/dt, section 2): a lone population must move
one cell per step along its velocity (Eq. 3-stencil-d2q5), wrap on periodic sides,
come back mirrored from a wall, be copied at an outflow side and be replaced by the
inflow equilibrium at an inflow side.  A lake at rest must stay exactly at rest.
"""

import itertools

import numpy as np
import pytest

import oracle
from oracle import INFLOW, OUTFLOW, PERIODIC, WALL
from paper_1401_0427_gb300 import inputs

# velocity of each 2D population in lattice units (section 3, D2Q5 stencil)
EX = [0, 1, 0, -1, 0, 1, 0, -1, 0, 1, 0, -1, 0]
EY = [0, 0, 1, 0, -1, 0, 1, 0, -1, 0, 1, 0, -1]


def _background(nx, ny):
    """Uniform populations of a lake of depth 1 (f1..f4 = 1/4, the rest 0); with s = 0
    they stream onto themselves on periodic, wall and outflow sides.  Dyadic values keep
    (background + spike) - background exact."""
    B = np.zeros((13, ny, nx))
    B[1:5] = 0.25
    return B


def _one_step_pure(F, nx, ny, bc, inflow=None):
    """One pure-streaming step (s = 0) of the perturbation F on top of the background:
    the collision needs h > 0 everywhere even when it changes nothing."""
    B = _background(nx, ny)
    return oracle.run_2d(B + F, 1, oracle.params(nx, ny, s=0.0, bc=bc, inflow=inflow)) - B


@pytest.mark.parametrize("pop", range(13))
def test_lone_population_moves_along_its_velocity(pop):
    nx, ny = 6, 5
    for (i, j) in [(2, 3), (0, 0), (5, 4)]:
        F = np.zeros((13, ny, nx))
        F[pop, j, i] = 1.0
        out = _one_step_pure(F, nx, ny, (PERIODIC,) * 4)
        want = np.zeros_like(F)
        want[pop, (j + EY[pop]) % ny, (i + EX[pop]) % nx] = 1.0
        assert np.array_equal(out, want)


# mirror partner across an x-wall / y-wall and the sign of the reflected value:
# f keeps its sign, the momentum family normal to the wall changes sign.
MIRROR_X = {1: (3, 1), 3: (1, 1), 5: (7, -1), 7: (5, -1), 9: (11, 1), 11: (9, 1)}
MIRROR_Y = {2: (4, 1), 4: (2, 1), 6: (8, 1), 8: (6, 1), 10: (12, -1), 12: (10, -1)}


@pytest.mark.parametrize("side", range(4))
def test_wall_reflects_outgoing_population(side):
    nx, ny = 5, 4
    bc = [WALL] * 4  # a periodic partner side would also wrap the spike around
    table = MIRROR_X if side < 2 else MIRROR_Y
    # populations leaving through this side
    outgoing = [p for p in table if (EX[p], EY[p]) == [(-1, 0), (1, 0), (0, -1), (0, 1)][side]]
    assert len(outgoing) == 3
    for pop in outgoing:
        i = {0: 0, 1: nx - 1}.get(side, 2)
        j = {2: 0, 3: ny - 1}.get(side, 1)
        F = np.zeros((13, ny, nx))
        F[pop, j, i] = 0.75
        out = _one_step_pure(F, nx, ny, bc)
        partner, sign = table[pop]
        want = np.zeros_like(F)
        want[partner, j, i] = sign * 0.75
        assert np.array_equal(out, want), (side, pop)


@pytest.mark.parametrize("side", range(4))
def test_outflow_copies_boundary_cell(side):
    nx, ny = 5, 4
    bc = [OUTFLOW] * 4
    incoming = [p for p in range(13) if (EX[p], EY[p]) == [(1, 0), (-1, 0), (0, 1), (0, -1)][side]]
    for pop in incoming:
        i = {0: 0, 1: nx - 1}.get(side, 3)
        j = {2: 0, 3: ny - 1}.get(side, 2)
        F = np.zeros((13, ny, nx))
        F[pop, j, i] = 0.5
        out = _one_step_pure(F, nx, ny, bc)
        want = np.zeros_like(F)
        want[pop, j, i] = 0.5  # the ghost copy of the boundary cell comes back in
        want[pop, j + EY[pop], i + EX[pop]] = 0.5  # and the population moves on inside
        assert np.array_equal(out, want), (side, pop)


@pytest.mark.parametrize("side", range(4))
def test_inflow_injects_equilibrium(side):
    nx, ny = 4, 3
    bc = [PERIODIC] * 4
    bc[side] = INFLOW
    w_in = (1.7, 0.3, -0.2)
    inflow = [None] * 4
    inflow[side] = w_in
    B = _background(nx, ny)
    out = oracle.run_2d(B, 1, oracle.params(nx, ny, s=0.0, bc=bc, inflow=inflow))
    feq = oracle.equilibrium_2d([w_in[0]], [w_in[1]], [w_in[2]], oracle.params(1, 1))[:, 0, 0]
    incoming = [p for p in range(13) if (EX[p], EY[p]) == [(1, 0), (-1, 0), (0, 1), (0, -1)][side]]
    want = B.copy()
    for pop in incoming:
        if side == 0:
            want[pop, :, 0] = feq[pop]
        elif side == 1:
            want[pop, :, nx - 1] = feq[pop]
        elif side == 2:
            want[pop, 0, :] = feq[pop]
        else:
            want[pop, ny - 1, :] = feq[pop]
    assert np.array_equal(out, want)


@pytest.mark.parametrize("side", range(2))
def test_inflow_injects_equilibrium_1d(side):
    """1D: with s = 0 the populations entering through an INFLOW side (f+ and g+ at x-,
    f- and g- at x+) are the equilibrium of the prescribed state W_in = (h, q), whose
    closed form (section 2) is written out here: f+- = (h - a kappa)/2 +- q/(2 lam),
    g+- = q/2 +- (q u + g h^2/2)/(2 lam), kappa = h/2 - u^2/(4g)."""
    n, lam, a, g = 5, 8.0, 0.15, 1.0
    bc = [OUTFLOW, OUTFLOW]
    bc[side] = INFLOW
    h, q = 1.7, 0.3
    inflow = [None] * 4
    inflow[side] = (h, q, 0.0)
    B = oracle.equilibrium_1d(np.ones(n), np.zeros(n), oracle.params(n, a=a))  # a lake of depth 1
    out = oracle.run_1d(B, 1, oracle.params(n, a=a, s=0.0, bc=bc, inflow=inflow))
    u = q / h
    kap = h / 2 - u * u / (4 * g)
    feq = [a * kap, (h - a * kap) / 2 + q / (2 * lam), (h - a * kap) / 2 - q / (2 * lam),
           q / 2 + (q * u + g * h * h / 2) / (2 * lam), q / 2 - (q * u + g * h * h / 2) / (2 * lam)]
    cell, incoming = (0, (1, 3)) if side == 0 else (n - 1, (2, 4))
    for pop in incoming:
        assert out[pop, cell] == pytest.approx(feq[pop], rel=1e-14, abs=1e-15)
    want = B.copy()
    for pop in incoming:
        want[pop, cell] = out[pop, cell]
    assert np.array_equal(out, want)  # every other population streamed onto the lake's own values


def test_pure_streaming_periodic_returns_after_n_steps():
    nx, ny = 7, 5
    F = inputs.random_populations(13, ny, nx, seed=41)
    p = oracle.params(nx, ny, s=0.0)
    assert np.array_equal(oracle.run_2d(F, nx * ny, p), F)  # every shift returns after lcm | nx*ny
    assert not np.array_equal(oracle.run_2d(F, 1, p), F)


def test_pure_streaming_walled_box_returns_after_2n_steps():
    n = 6
    F = inputs.random_populations(13, n, n, seed=42)
    p = oracle.params(n, n, s=0.0, bc=(WALL,) * 4)
    assert np.array_equal(oracle.run_2d(F, 2 * n, p), F)
    assert not np.array_equal(oracle.run_2d(F, n, p), F)


def test_pure_streaming_1d_walls_and_periodic():
    n = 9
    F = inputs.random_populations(5, 1, n, seed=43).reshape(5, n)
    assert np.array_equal(oracle.run_1d(F, 2 * n, oracle.params(n, s=0.0, bc=(WALL, WALL))), F)
    assert np.array_equal(oracle.run_1d(F, n, oracle.params(n, s=0.0, bc=(PERIODIC, PERIODIC))), F)
    # one step against the left wall: f- at cell 0 comes back as f+, g- as -g+
    B = np.zeros((5, n))
    B[1:3] = 0.5  # depth-1 background so that the (identity) collision is defined
    G = np.zeros((5, n))
    G[2, 0], G[4, 0] = 0.25, 0.125
    out = oracle.run_1d(B + G, 1, oracle.params(n, s=0.0, bc=(WALL, WALL))) - B
    want = np.zeros((5, n))
    want[1, 0], want[3, 0] = 0.25, -0.125
    assert np.array_equal(out, want)


@pytest.mark.parametrize("side", range(2))
def test_outflow_copies_boundary_cell_1d(side):
    """1D, s = 0: a population entering through an OUTFLOW side is the boundary cell's own
    value of it (the ghost is a copy of that cell), here a spike of 0.25 on f+ or g+ at x-
    and on f- or g- at x+, which also moves on inside."""
    n = 6
    B = np.zeros((5, n))
    B[1:3] = 0.5  # depth-1 background so that the (identity) collision is defined
    cell, step, incoming = (0, 1, (1, 3)) if side == 0 else (n - 1, -1, (2, 4))
    for pop in incoming:
        G = np.zeros((5, n))
        G[pop, cell] = 0.25
        out = oracle.run_1d(B + G, 1, oracle.params(n, s=0.0, bc=(OUTFLOW, OUTFLOW))) - B
        want = np.zeros((5, n))
        want[pop, cell] = 0.25  # the ghost copy comes back in
        want[pop, cell + step] = 0.25  # and the spike moves on
        assert np.array_equal(out, want), (side, pop)


@pytest.mark.parametrize("h0", [1.0, 2.0, 0.5])
@pytest.mark.parametrize("bcs", [(PERIODIC,) * 4, (WALL,) * 4, (OUTFLOW,) * 4, (WALL, OUTFLOW, PERIODIC, PERIODIC)])
def test_lake_at_rest_stays_exactly_at_rest(h0, bcs):
    nx, ny = 9, 7
    p = oracle.params(nx, ny, bc=bcs)
    F = oracle.equilibrium_2d(np.full(nx * ny, h0), np.zeros(nx * ny), np.zeros(nx * ny), p)
    out = oracle.run_2d(F, 50, p)
    rho, qx, qy = oracle.moments_2d(out, p)
    assert np.array_equal(rho, np.full((ny, nx), h0))
    assert np.array_equal(qx, np.zeros((ny, nx))) and np.array_equal(qy, np.zeros((ny, nx)))
    assert np.array_equal(out, F)


def test_lake_at_rest_with_matching_inflow_stays_at_rest():
    nx, ny, h0 = 8, 6, 1.0
    p = oracle.params(nx, ny, bc=(INFLOW, INFLOW, INFLOW, INFLOW), inflow=[(h0, 0.0, 0.0)] * 4)
    F = oracle.equilibrium_2d(np.full(nx * ny, h0), np.zeros(nx * ny), np.zeros(nx * ny), p)
    assert np.array_equal(oracle.run_2d(F, 30, p), F)


def test_lake_at_rest_1d():
    n = 33
    for bc in itertools.product([PERIODIC, WALL, OUTFLOW], repeat=2):
        if (bc[0] == PERIODIC) != (bc[1] == PERIODIC):
            continue
        p = oracle.params(n, a=0.15, bc=bc)
        F = oracle.equilibrium_1d(np.ones(n), np.zeros(n), p)
        assert np.array_equal(oracle.run_1d(F, 40, p), F)


@pytest.mark.parametrize("bc", [(PERIODIC,) * 4, (WALL, OUTFLOW, INFLOW, WALL)], ids=["P", "WOIW"])
def test_separate_collide_and_stream_make_one_step(bc):
    """The stand-alone collide and stream entry points, applied in turn, give one step of
    the (pinned) run, bit for bit, in 1D and 2D."""
    inflow = [(1.2, 0.1, -0.05)] * 4
    nx, ny = 7, 5
    F = inputs.random_populations(13, ny, nx, seed=71)
    p = oracle.params(nx, ny, bc=bc, inflow=inflow)
    assert np.array_equal(oracle.stream_2d(oracle.collide_2d(F, p), p), oracle.run_2d(F, 1, p))
    F1 = inputs.random_populations(5, 1, nx, seed=72).reshape(5, nx)
    p1 = oracle.params(nx, a=0.15, bc=bc[:2], inflow=inflow)
    assert np.array_equal(oracle.stream_1d(oracle.collide_1d(F1, p1), p1), oracle.run_1d(F1, 1, p1))
