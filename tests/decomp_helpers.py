"""A host stand-in for lbm_sw.Simulation in the decomposition tests: the same methods, with
the FP64 oracle advancing the band (test infrastructure: the product's decomposition never
imports the oracle; the tests hand this object to it as the band's stepper).

It keeps the oracle's pre-collision populations; the rows it exchanges are in that form on
every band, which carries the same information as the library's post-collision rows (the
collision is local to a cell)."""

from __future__ import annotations

from types import SimpleNamespace

import numpy as np

import oracle


class OracleStepper:
    def __init__(self, nx, ny, *, bc, a=0.05, inflow=None):
        self.nx, self.ny, self.q, self.dtype = nx, ny, 13, np.float64
        self.p = oracle.params(nx, ny, a=a, bc=bc, inflow=inflow)
        self.F = None
        self.steps = 0

    def info(self):
        return SimpleNamespace(steps_per_launch=1)

    def set_state(self, h, hu, hv):
        self.F = oracle.equilibrium_2d(h, hu, hv, self.p)

    def step(self, n):
        self.F = oracle.run_2d(self.F, int(n), self.p)
        self.steps += int(n)

    def get_rows_into(self, y0, n, out):
        rows = self.F[:, y0:y0 + n, :]
        if hasattr(out, "numpy"):
            out.numpy()[...] = rows
        else:
            out[...] = rows

    def set_rows(self, y0, n, src):
        self.F[:, y0:y0 + n, :] = src.numpy() if hasattr(src, "numpy") else src

    def moments(self):
        return oracle.moments_2d(self.F, self.p)

    def diagnostics_rows(self, y0, n, raise_unstable=True):
        h, hu, hv = (x[y0:y0 + n] for x in self.moments())
        bad = int(np.count_nonzero(~np.isfinite(h) | (h <= 0)))
        return float(h.sum()), float(hu.sum()), float(hv.sum()), float(h.min()), (0 if bad == 0 else -3)
