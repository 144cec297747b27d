"""Seeded synthetic inputs for the shallow-water lattice Boltzmann workloads.

This module holds no arithmetic of the scheme: it draws random numbers and lays
out initial depth/discharge fields (or raw populations) for the workloads of the
paper (dam-break shock tube of section 2, shock reflection and unsteady 2D flows
of section 4) at the sizes of the benchmark.  Both the CUDA path and the CPU
oracle receive exactly these arrays, so the two sides share inputs and nothing
else.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: output k of stream ``seed`` is ``mix(seed + (k + 1) * gamma)``.
Every field is a pure function of (seed, index), so any sub-block can be
regenerated without drawing the rest.
"""

from __future__ import annotations

import math

import numpy as np

BASE_SEED = 0x14010427
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset + count - 1`` of the SplitMix64 stream ``seed``."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int, lo: float = 0.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    """``count`` doubles uniform in [lo, hi): the top 53 bits of each output."""
    u = (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def stream_seed(config: int, sub: int = 0) -> int:
    """Seed of stream ``sub`` of workload ``config`` (base 0x14010427)."""
    return (BASE_SEED + (config << 32) + (sub << 48)) & 0xFFFFFFFFFFFFFFFF


def cell_centres(n: int) -> np.ndarray:
    """Centres (i + 1/2)/n of n cells on [0, 1]."""
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def centred_offsets(n: int) -> np.ndarray:
    """Offsets of the cell centres from 1/2, written (2i + 1 - n)/(2n) so that the
    offsets of mirror-image cells are exact negatives of each other."""
    return (2.0 * np.arange(n, dtype=np.float64) + 1.0 - n) / (2.0 * n)


# ------------------------------------------------------------------ 1D fields
def dam_break_1d(n: int, h_left: float = 2.0, h_right: float = 1.0, x0: float = 0.5):
    """Riemann problem at rest: h = h_left for x < x0 else h_right, q = 0, on [0, 1]."""
    x = cell_centres(n)
    h = np.where(x < x0, h_left, h_right).astype(np.float64)
    return h, np.zeros(n)


# ------------------------------------------------------------------ 2D fields
def shock_speed_state(h_left: float, h_right: float, g: float = 1.0) -> float:
    """Velocity behind a shock running into still water of depth ``h_right`` with
    depth ``h_left`` behind it (Rankine-Hugoniot for shallow water)."""
    return (h_left - h_right) * math.sqrt(g * (h_left + h_right) / (2.0 * h_left * h_right))


def planar_shock_2d(nx: int, ny: int, h_left: float = 2.0, h_right: float = 1.0,
                    x0: float = 0.5, g: float = 1.0):
    """A planar shock at x = x0 moving in +x: (h_left, u_left) behind, (h_right, 0) ahead."""
    u_left = shock_speed_state(h_left, h_right, g)
    x = cell_centres(nx)[None, :] * np.ones((ny, 1))
    behind = x < x0
    h = np.where(behind, h_left, h_right)
    hu = np.where(behind, h_left * u_left, 0.0)
    return h, hu, np.zeros((ny, nx))


def circular_dam_break_2d(n: int, seed: int | None = None, h_in: float = 2.0, h_out: float = 1.0,
                          radius: float = 0.2, perturbation: float = 1e-3):
    """Column of depth ``h_in`` for r < radius (strictly, at cell centres) around the
    centre of the unit square, ``h_out`` elsewhere, at rest, plus a uniform
    perturbation in [-perturbation, +perturbation) of h drawn from ``seed`` (none if
    seed is None).  Returns (h, hu, hv) as [n][n] arrays, x fastest."""
    o = centred_offsets(n)
    r2 = o[None, :] * o[None, :] + o[:, None] * o[:, None]
    h = np.where(r2 < radius * radius, h_in, h_out).astype(np.float64)
    if seed is not None and perturbation != 0.0:
        h = h + uniform(seed, n * n, -perturbation, perturbation).reshape(n, n)
    z = np.zeros((n, n))
    return h, z, z.copy()


def gaussian_bumps_2d(n: int, seed: int, count: int = 8, depth: float = 1.0,
                      amp=(0.05, 0.3), sigma=(0.03, 0.1)):
    """Depth ``depth`` plus ``count`` Gaussian bumps with periodic distance on the unit
    square: amplitudes, widths and centres drawn (in that order per bump) from ``seed``."""
    r = uniform(seed, 4 * count).reshape(count, 4)
    c = cell_centres(n)
    h = np.full((n, n), depth)
    for k in range(count):
        a = amp[0] + (amp[1] - amp[0]) * r[k, 0]
        s = sigma[0] + (sigma[1] - sigma[0]) * r[k, 1]
        dx = np.abs(c - r[k, 2]); dx = np.minimum(dx, 1.0 - dx)
        dy = np.abs(c - r[k, 3]); dy = np.minimum(dy, 1.0 - dy)
        h += a * np.exp(-(dy[:, None] ** 2 + dx[None, :] ** 2) / (2.0 * s * s))
    z = np.zeros((n, n))
    return h, z, z.copy()


def batched_instances(count: int = 256, seed: int | None = None, side=(64, 1024),
                      h_in=(1.5, 4.0), radius=(0.1, 0.3)):
    """Instance table of the batched dam-breaks: per instance (side, h_in, radius),
    drawn in that order; side uniform over the integers side[0]..side[1]."""
    seed = stream_seed(4) if seed is None else seed
    r = uniform(seed, 3 * count).reshape(count, 3)
    out = []
    for k in range(count):
        n = side[0] + min(int(r[k, 0] * (side[1] - side[0] + 1)), side[1] - side[0])
        out.append((n, h_in[0] + (h_in[1] - h_in[0]) * r[k, 1],
                    radius[0] + (radius[1] - radius[0]) * r[k, 2]))
    return out


# --------------------------------------------------------- raw populations
def random_populations(q: int, ny: int, nx: int, seed: int) -> np.ndarray:
    """Arbitrary (non-equilibrium) populations with positive depth: the mass family
    (the first 5 planes in 2D, the first 3 in 1D) uniform in [0.05, 0.45), the
    momentum families uniform in [-0.1, 0.1)."""
    nmass = 5 if q == 13 else 3
    n = ny * nx
    F = np.empty((q, ny, nx))
    F[:nmass] = uniform(seed, nmass * n, 0.05, 0.45).reshape(nmass, ny, nx)
    F[nmass:] = uniform(seed, (q - nmass) * n, -0.1, 0.1, offset=nmass * n).reshape(q - nmass, ny, nx)
    return F


def random_states(n: int, seed: int, h=(0.5, 3.0), speed: float = 0.6):
    """``n`` admissible states (h, h u, h v) with |u|, |v| < speed."""
    r = uniform(seed, 3 * n).reshape(3, n)
    hh = h[0] + (h[1] - h[0]) * r[0]
    return hh, hh * speed * (2 * r[1] - 1), hh * speed * (2 * r[2] - 1)


def random_obstacles(ny: int, nx: int, seed: int, fraction: float = 0.15) -> np.ndarray:
    """Solid-cell mask ``[ny][nx]`` (uint8, 1 = solid): each cell solid with probability
    ``fraction``."""
    return (uniform(seed, ny * nx).reshape(ny, nx) < fraction).astype(np.uint8)


def emery_step(nx: int, ny: int, froude: float = 3.0, h0: float = 1.0, g: float = 1.0,
               step_x: float = 0.6, step_h: float = 0.2):
    """Forward-facing step in a channel of height 1 and length nx / ny (cells of side 1 / ny):
    the step's front face stands at x = step_x and it fills [step_x, nx / ny] x [0, step_h]
    (cells whose centre lies there are solid).  The channel starts filled with the inflow
    state: depth h0, velocity froude sqrt(g h0) along x.

    Returns (solid, (h, hu, hv), inflow_state)."""
    xc = (np.arange(nx, dtype=np.float64) + 0.5) / ny
    yc = (np.arange(ny, dtype=np.float64) + 0.5) / ny
    X, Y = np.meshgrid(xc, yc)
    solid = ((X > step_x) & (Y < step_h)).astype(np.uint8)
    u = froude * math.sqrt(g * h0)
    h = np.full((ny, nx), h0)
    return solid, (h, h * u, np.zeros((ny, nx))), (h0, h0 * u, 0.0)
