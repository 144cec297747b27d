"""The exact solutions that the experiments module reports next to the GPU runs agree
with the independent closed forms of the tests (CPU only)."""

import math

import numpy as np

from paper_1401_0427_gb300 import experiments as ex

from exact import oblique_jump_residual, stoker


def test_stoker_matches_the_test_closed_form():
    for hr in (1.0, 0.5, 0.2):
        a = ex.stoker(2.0, hr)
        b = stoker(2.0, hr)
        assert abs(a[0] - b[0]) < 1e-13 and abs(a[1] - b[1]) < 1e-13 and abs(a[4] - b[2]) < 1e-12


def test_reflection_exact_solution_is_a_rankine_hugoniot_pattern():
    ang = ex.reflected_shock_angle()
    assert abs(math.tan(ang) - 1.25) < 1e-9 and 0 < ang < math.pi / 2
    assert np.abs(oblique_jump_residual(ex.REFLECTION_TOP, ex.REFLECTION_RIGHT, ang)).max() < 1e-12
    assert np.abs(oblique_jump_residual(ex.REFLECTION_LEFT, ex.REFLECTION_TOP, ex.INCIDENT_ANGLE)).max() < 1e-13
    xc = (np.arange(140) + 0.5) / 80
    yc = (np.arange(80) + 0.5) / 80
    h, hu, hv = ex.reflection_exact(xc, yc)
    assert set(np.unique(h)) == {ex.REFLECTION_LEFT[0], ex.REFLECTION_TOP[0], ex.REFLECTION_RIGHT[0]}
    assert h[0, 0] == ex.REFLECTION_LEFT[0] and h[-1, 70] == ex.REFLECTION_TOP[0] and h[2, -1] == ex.REFLECTION_RIGHT[0]
    assert np.all(hv[h == ex.REFLECTION_RIGHT[0]] == 0.0)
