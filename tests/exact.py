"""Closed-form solutions of the shallow-water equations used to pin the oracle.

These are textbook results, independent of the lattice Boltzmann scheme:

* Stoker's wet dam-break (Riemann problem at rest, h_left > h_right > 0): a left
  rarefaction fan and a right shock around a middle state (h*, u*) that solves
      2 (sqrt(g h_l) - sqrt(g h*)) = (h* - h_r) sqrt(g (h* + h_r) / (2 h* h_r)).
* Rankine-Hugoniot jump across a shock reflected by a wall: a state (h1, u1 > 0)
  meeting a wall at rest turns into (h2, 0) behind a shock of speed S < 0 with
      S (h2 - h1) = -h1 u1,   g h2^2/2 - h1 u1^2 - g h1^2/2 = -S h1 u1.
* Rankine-Hugoniot conditions across a stationary oblique shock (continuity of the
  normal mass flux, of the normal momentum flux and of the tangential velocity).
"""

from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def stoker(h_left: float, h_right: float, g: float = 1.0):
    """Middle state and wave speeds of the wet dam-break: (h*, u*, shock speed,
    fan head speed, fan tail speed)."""
    cl = math.sqrt(g * h_left)

    def mismatch(hs):
        return 2.0 * (cl - math.sqrt(g * hs)) - (hs - h_right) * math.sqrt(g * (hs + h_right) / (2.0 * hs * h_right))

    hs = brentq(mismatch, h_right, h_left, xtol=1e-15, rtol=1e-15, maxiter=200)
    us = 2.0 * (cl - math.sqrt(g * hs))
    shock = hs * us / (hs - h_right)
    return hs, us, shock, -cl, us - math.sqrt(g * hs)


def stoker_profile(x: np.ndarray, t: float, h_left: float, h_right: float, x0: float = 0.5, g: float = 1.0):
    """Exact (h, u) at positions x and time t > 0 of the dam-break released at x0."""
    hs, us, shock, head, tail = stoker(h_left, h_right, g)
    cl = math.sqrt(g * h_left)
    xi = (np.asarray(x, dtype=np.float64) - x0) / t
    h = np.where(xi < head, h_left,
                 np.where(xi < tail, (2.0 * cl - xi) ** 2 / (9.0 * g),
                          np.where(xi < shock, hs, h_right)))
    u = np.where(xi < head, 0.0,
                 np.where(xi < tail, 2.0 / 3.0 * (cl + xi),
                          np.where(xi < shock, us, 0.0)))
    return h, u


def wall_reflection(h1: float, u1: float, g: float = 1.0):
    """Depth h2 at rest behind the shock reflected by a wall, and that shock's speed."""

    def mismatch(h2):
        s = -h1 * u1 / (h2 - h1)
        return (g * h2 * h2 / 2.0) - (h1 * u1 * u1 + g * h1 * h1 / 2.0) + s * h1 * u1

    h2 = brentq(mismatch, h1 * (1 + 1e-12), 100.0 * h1, xtol=1e-15, rtol=1e-15, maxiter=200)
    return h2, -h1 * u1 / (h2 - h1)


def oblique_jump_residual(a, b, angle: float, g: float = 1.0):
    """Residuals of the Rankine-Hugoniot conditions between states a = (h, u, v) and
    b across a stationary straight shock whose line makes ``angle`` with the x axis:
    (normal mass flux, normal momentum flux, tangential velocity)."""
    t = np.array([math.cos(angle), math.sin(angle)])
    n = np.array([-t[1], t[0]])
    ha, ua = a[0], np.array(a[1:3])
    hb, ub = b[0], np.array(b[1:3])
    una, unb = ua @ n, ub @ n
    return np.array([
        ha * una - hb * unb,
        ha * una * una + g * ha * ha / 2.0 - (hb * unb * unb + g * hb * hb / 2.0),
        ua @ t - ub @ t,
    ])
