"""Helpers shared by the GPU parity tests: run a case through the C ABI and the same
case through the oracle, from the same seeded inputs.

Tolerances (written into the tests that use them):
  FP64: max |gpu - oracle| / max |oracle| <= 1e-12 (the stated bar for FP64).
  FP32: relative L1 of h, sum |h_gpu - h_oracle| / sum |h_oracle| <= 1e-5 (the stated
        bar), and, for runs of a few steps, an element-wise bound of 1e-5 of the field
        scale: each step rounds ~25 dependent FP32 operations (unit roundoff 6e-8).
"""

from __future__ import annotations

import numpy as np

import oracle
from paper_1401_0427_gb300 import lbm_sw

FP64_TOL = 1e-12
FP32_L1_TOL = 1e-5
FP32_ELEM_TOL = 1e-5

BC_NAMES = {lbm_sw.PERIODIC: "P", lbm_sw.WALL: "W", lbm_sw.OUTFLOW: "O", lbm_sw.INFLOW: "I"}


def torch_stream():
    import torch

    return torch.cuda.current_stream().cuda_stream


def oracle_params(nx, ny, dim, bc, inflow, a, lam=8.0, s=1.8, solid=None):
    return oracle.params(nx, ny, a=a, lam=lam, s=s, bc=bc, inflow=inflow, solid=solid)


def oracle_post(F0: np.ndarray, steps: int, p, dim: int) -> np.ndarray:
    """Post-collision populations after ``steps`` steps from pre-collision F0."""
    if dim == 1:
        return oracle.collide_1d(oracle.run_1d(F0.reshape(5, -1), steps, p), p).reshape(F0.shape)
    return oracle.collide_2d(oracle.run_2d(F0, steps, p), p)


def gpu_post(F0: np.ndarray, steps: int, *, dim: int, precision: int, bc, inflow, a, kernel=lbm_sw.KERNEL_AUTO,
             lam=8.0, s=1.8, graph_chunk=0, mrt_rates=None, solid=None) -> np.ndarray:
    q, ny, nx = F0.shape
    with lbm_sw.Simulation(nx, ny, dim=dim, precision=precision, bc=bc, inflow=inflow, a=a, lam=lam, s=s,
                           kernel=kernel, stream=torch_stream(), graph_chunk=graph_chunk) as sim:
        if mrt_rates is not None:
            sim.set_relaxation(mrt_rates)
        if solid is not None:
            sim.set_obstacle(solid)
        sim.set_populations(F0, form=lbm_sw.PRE_COLLISION)
        sim.step(steps)
        return sim.populations().astype(np.float64)


def rel_max(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_l1(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.abs(a - b).sum() / np.abs(b).sum())
