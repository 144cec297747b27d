"""Pins of the oracle's obstacles (solid cells inside the domain, mirror walls on their faces).

The paper's second 2D test (section 4, Emery's forward-facing step) needs walls inside the
domain; the paper gives the wall rule only for domain sides.  The reading: a face between a
fluid and a solid cell is a wall with the same mirror rule as a domain side.  Pinned by:

* equivalence with the domain-side wall: a fluid region closed by solid columns or rows
  evolves exactly like a domain of the same size with WALL sides, including through a
  periodic side (bit for bit: the same operations on the same values);
* conservation: the fluid's total depth is conserved to round-off in a box with scattered
  obstacles, and solid cells never change;
* a lake at rest around obstacles stays exactly at rest;
* symmetry: a mirror-symmetric obstacle in a mirror-symmetric flow keeps the symmetry bit
  for bit.
"""

import numpy as np
import pytest

import oracle
from oracle import INFLOW, OUTFLOW, PERIODIC, WALL
from paper_1401_0427_gb300 import inputs

INFLOW_STATES = [(1.3, 0.2, -0.1), (0.9, -0.15, 0.05), (1.1, 0.05, 0.12), (1.2, -0.08, -0.2)]


def _embed(F, pad_x=(0, 0), pad_y=(0, 0), fill=None):
    """Place F ([13][ny][nx]) inside a larger grid; the new cells get `fill` populations."""
    q, ny, nx = F.shape
    out = np.empty((q, ny + sum(pad_y), nx + sum(pad_x)))
    out[...] = 0.0 if fill is None else fill[:, None, None]
    out[:, pad_y[0]:pad_y[0] + ny, pad_x[0]:pad_x[0] + nx] = F
    return out


@pytest.mark.parametrize("ybc", [PERIODIC, WALL, OUTFLOW, INFLOW])
def test_solid_columns_equal_x_walls(ybc):
    nx, ny, steps = 9, 7, 6
    F0 = inputs.random_populations(13, ny, nx, seed=800 + ybc)
    ref = oracle.run_2d(F0, steps, oracle.params(nx, ny, bc=(WALL, WALL, ybc, ybc), inflow=INFLOW_STATES))
    fill = inputs.random_populations(13, 1, 1, seed=801)[:, 0, 0]
    big = _embed(F0, pad_x=(1, 1), fill=fill)
    solid = np.zeros((ny, nx + 2), dtype=np.uint8)
    solid[:, 0] = solid[:, -1] = 1
    p = oracle.params(nx + 2, ny, bc=(OUTFLOW, INFLOW, ybc, ybc), inflow=INFLOW_STATES, solid=solid)
    got = oracle.run_2d(big, steps, p)
    assert np.array_equal(got[:, :, 1:-1], ref)
    assert np.array_equal(got[:, :, 0], big[:, :, 0]) and np.array_equal(got[:, :, -1], big[:, :, -1])


@pytest.mark.parametrize("xbc", [PERIODIC, WALL, OUTFLOW, INFLOW])
def test_solid_rows_equal_y_walls(xbc):
    nx, ny, steps = 6, 8, 6
    F0 = inputs.random_populations(13, ny, nx, seed=810 + xbc)
    ref = oracle.run_2d(F0, steps, oracle.params(nx, ny, bc=(xbc, xbc, WALL, WALL), inflow=INFLOW_STATES))
    big = _embed(F0, pad_y=(1, 1))
    solid = np.zeros((ny + 2, nx), dtype=np.uint8)
    solid[0, :] = solid[-1, :] = 1
    p = oracle.params(nx, ny + 2, bc=(xbc, xbc, OUTFLOW, WALL), inflow=INFLOW_STATES, solid=solid)
    got = oracle.run_2d(big, steps, p)
    assert np.array_equal(got[:, 1:-1, :], ref)


def test_one_solid_column_across_a_periodic_side():
    """Periodic in x with a single solid column 0: cells 1 .. nx see walls on both sides,
    the right one reached through the periodic wrap."""
    nx, ny, steps = 10, 5, 8
    F0 = inputs.random_populations(13, ny, nx, seed=820)
    ref = oracle.run_2d(F0, steps, oracle.params(nx, ny, bc=(WALL, WALL, PERIODIC, PERIODIC)))
    big = _embed(F0, pad_x=(1, 0))
    solid = np.zeros((ny, nx + 1), dtype=np.uint8)
    solid[:, 0] = 1
    got = oracle.run_2d(big, steps, oracle.params(nx + 1, ny, solid=solid))
    assert np.array_equal(got[:, :, 1:], ref)


def test_solid_row_across_a_periodic_side():
    nx, ny, steps = 5, 9, 8
    F0 = inputs.random_populations(13, ny, nx, seed=821)
    ref = oracle.run_2d(F0, steps, oracle.params(nx, ny, bc=(PERIODIC, PERIODIC, WALL, WALL)))
    big = _embed(F0, pad_y=(0, 1))
    solid = np.zeros((ny + 1, nx), dtype=np.uint8)
    solid[-1, :] = 1
    got = oracle.run_2d(big, steps, oracle.params(nx, ny + 1, solid=solid))
    assert np.array_equal(got[:, :-1, :], ref)


def _scattered_solid(nx, ny, seed, frac=0.15):
    return inputs.random_obstacles(ny, nx, seed=seed, fraction=frac)


@pytest.mark.parametrize("bc", [(WALL,) * 4, (PERIODIC,) * 4, (PERIODIC, PERIODIC, WALL, WALL)])
def test_fluid_mass_is_conserved_and_solid_cells_do_not_change(bc):
    nx, ny = 24, 18
    solid = _scattered_solid(nx, ny, 830)
    h, qx, qy = (w.reshape(ny, nx) for w in inputs.random_states(ny * nx, seed=831))
    p = oracle.params(nx, ny, bc=bc, solid=solid)
    F0 = oracle.equilibrium_2d(h, qx, qy, p)
    F = oracle.run_2d(F0, 60, p)
    fluid = solid == 0
    m0 = oracle.moments_2d(F0, p)[0][fluid].sum()
    m1 = oracle.moments_2d(F, p)[0][fluid].sum()
    assert abs(m1 - m0) <= 1e-12 * m0
    assert np.array_equal(F[:, solid != 0], F0[:, solid != 0])


def test_lake_at_rest_around_obstacles_stays_at_rest():
    nx, ny = 20, 14
    solid = _scattered_solid(nx, ny, 840, frac=0.2)
    one, zero = np.full((ny, nx), 1.3), np.zeros((ny, nx))
    for bc in [(WALL,) * 4, (PERIODIC,) * 4]:
        p = oracle.params(nx, ny, bc=bc, solid=solid)
        F0 = oracle.equilibrium_2d(one, zero, zero, p)
        F = oracle.run_2d(F0, 25, p)
        np.testing.assert_allclose(F, F0, rtol=0, atol=1e-15)
        h, qx, qy = oracle.moments_2d(F, p)
        assert np.abs(qx).max() <= 1e-15 and np.abs(qy).max() <= 1e-15


def test_symmetric_obstacle_keeps_mirror_symmetry():
    """A block centred in x in a dam-break centred in x: the field stays x-mirror symmetric
    (h even, hu odd) bit for bit."""
    nx, ny = 30, 20
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[6:10, 12:18] = 1
    x = (np.arange(nx) + 0.5) / nx - 0.5
    y = (np.arange(ny) + 0.5) / ny - 0.7
    X, Y = np.meshgrid(x, y)
    h = np.where(X * X + Y * Y < 0.04, 2.0, 1.0)
    z = np.zeros_like(h)
    p = oracle.params(nx, ny, bc=(WALL, WALL, WALL, WALL), solid=solid)
    F = oracle.run_2d(oracle.equilibrium_2d(h, z, z, p), 40, p)
    H, QX, QY = oracle.moments_2d(F, p)
    fluid = solid == 0
    assert np.array_equal(H[fluid], H[:, ::-1][fluid])
    assert np.array_equal(QX[fluid], -QX[:, ::-1][fluid])
    assert np.array_equal(QY[fluid], QY[:, ::-1][fluid])
    assert np.abs(QX[fluid]).max() > 1e-3  # the flow did reach the obstacle
