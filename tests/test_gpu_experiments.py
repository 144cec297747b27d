"""The paper's test cases on the GPU (the next rows after the hot path), against the oracle
and the exact solutions.

* Section 2 shock tube (80 points, rho_r = 0.5, a = 0.15, s = 1.8, lambda = 8): the GPU run
  equals the oracle's; L1 errors against Stoker's solution fall as the mesh is refined.
* The same Riemann problem with the 2D scheme on a grid uniform in y: rows stay equal bit
  for bit, the run equals the oracle's, and it converges toward Stoker's solution.
* Section 4 stationary shock reflection (printed states): the GPU run reaches a steady
  state equal to the oracle's, the plateau behind the reflected shock matches the printed
  right state, and the L1 error falls over the paper's three meshes.
"""


import numpy as np
import pytest

import oracle
from paper_1401_0427_gb300 import experiments as ex
from paper_1401_0427_gb300 import inputs

from gpu_helpers import FP64_TOL, rel_max, torch_stream

pytestmark = pytest.mark.gpu


def test_paper_shock_tube_80_points():
    r = ex.shock_tube(80, stream=torch_stream())
    p = oracle.params(80, a=0.15, bc=(oracle.WALL, oracle.WALL))
    h0, q0 = inputs.dam_break_1d(80, 2.0, 0.5)
    oh, oq = oracle.moments_1d(oracle.run_1d(oracle.equilibrium_1d(h0, q0, p), r["steps"], p), p)
    assert rel_max(r["h"], oh) <= FP64_TOL
    hs, us, *_ = ex.stoker(2.0, 0.5)
    mid = (r["x"] > 0.55) & (r["x"] < 0.72)
    assert np.all(np.abs(r["h"][mid] - hs) < 0.05 * hs) and np.all(np.abs(r["u"][mid] - us) < 0.05 * us)
    errs = [ex.shock_tube(n, stream=torch_stream())["l1_h"] for n in (80, 160, 320, 640, 1280)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_y_invariant_2d_dam_break():
    errs = []
    for n in (200, 400, 800, 1600):
        r = ex.dam_break_y_invariant(n, ny=4, stream=torch_stream())
        assert np.array_equal(r["h"], np.broadcast_to(r["h"][:1], r["h"].shape)) and np.all(r["hv"] == 0)
        errs.append(r["l1_h"])
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    n = 400
    r = ex.dam_break_y_invariant(n, ny=4, stream=torch_stream())
    p = oracle.params(n, 1, a=0.05, bc=(oracle.WALL, oracle.WALL, oracle.PERIODIC, oracle.PERIODIC))
    h1, q1 = inputs.dam_break_1d(n)
    oh = oracle.moments_2d(oracle.run_2d(oracle.equilibrium_2d(h1, q1, 0 * q1, p), r["steps"], p), p)[0]
    assert rel_max(r["h"][0], oh[0]) <= FP64_TOL


def test_stationary_shock_reflection():
    e = ex.oblique_shock_reflection(70, 40, stream=torch_stream())
    assert e["residuals"][-1][1] < 1e-10
    # the oracle reaches the same steady state
    nx, ny = 70, 40
    L, T = ex.REFLECTION_LEFT, ex.REFLECTION_TOP
    X, Y = np.meshgrid(e["x"], e["y"])
    up = Y < 1.0 - X
    W0 = (np.where(up, L[0], T[0]), np.where(up, L[0] * L[1], T[0] * T[1]), np.where(up, L[0] * L[2], T[0] * T[2]))
    inflow = [(L[0], L[0] * L[1], L[0] * L[2]), None, None, (T[0], T[0] * T[1], T[0] * T[2])]
    p = oracle.params(nx, ny, a=0.05, bc=(oracle.INFLOW, oracle.OUTFLOW, oracle.WALL, oracle.INFLOW), inflow=inflow)
    oh = oracle.moments_2d(oracle.run_2d(oracle.equilibrium_2d(*W0, p), e["steps"], p), p)[0]
    assert rel_max(e["h"], oh) <= 1e-11
    # the plateau behind the reflected shock is the printed right state
    R = ex.REFLECTION_RIGHT
    plateau = (X > 1.4) & (Y < 0.15)
    assert abs(e["h"][plateau].mean() - R[0]) < 1e-3 * R[0]
    assert abs((e["hu"][plateau] / e["h"][plateau]).mean() - R[1]) < 1e-3 * R[1]
    # far upstream of the (numerically smeared) incident shock the left state is untouched
    upstream = (X + Y < 0.6)
    assert np.all(np.abs(e["h"][upstream] - L[0]) < 1e-4)
    # the error falls over the paper's three meshes
    errs = [ex.oblique_shock_reflection(nx, ny, stream=torch_stream())["l1_h"] for nx, ny in ((35, 20), (70, 40), (140, 80))]
    assert errs[0] > errs[1] > errs[2], errs
