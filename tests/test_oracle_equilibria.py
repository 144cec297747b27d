"""Pins of the oracle's equilibria and collision against what the paper fixes.

* 1D (section 2): the potentials h_0^*, h_pm^* (Eqs. 2-potentiels-st-venant-1d and
  -suite) satisfy the Perthame-Bouchut identities (Eq. 2-perthame-bouchut-st-venant);
  the equilibria are their derivatives in (theta, beta), taken here by complex step
  on the potentials as printed, and their velocity moments are the physical fluxes.
* 2D (section 3): the 13 printed moment equilibria determine the 13 populations
  uniquely (the moment map is invertible), so checking all 13 pins every
  equilibrium.  Two printed lines are read as misprints: eps_rho^eq carries a
  factor a on its velocity term, and f_yy^eq = rho v^2 + p by symmetry with f_xx^eq.
* Collision (Eq. 2-relaxation): conservation of the conserved moments, s = 0 and
  s = 1 limits, MRT with equal rates equal to BGK, and MRT relaxing each printed
  moment at its own rate.
"""

import numpy as np
import pytest

import oracle
from paper_1401_0427_gb300 import inputs

G = 1.0


def _states(n, seed):
    return inputs.random_states(n, seed)


# --------------------------------------------------------------------- 1D
def _pot_1d(theta, beta, lam, a):
    """Potentials of section 2 as printed (K = 1/(2g))."""
    K = 1.0 / (2.0 * G)
    w2 = (theta + beta * beta / 2.0) ** 2
    h0 = a / 2.0 * K * theta * theta
    hp = K / 2.0 * w2 * (1.0 + beta / lam) - a * K / 4.0 * theta * theta
    hm = K / 2.0 * w2 * (1.0 - beta / lam) - a * K / 4.0 * theta * theta
    return h0, hp, hm


@pytest.mark.parametrize("a,lam", [(0.15, 8.0), (0.0, 8.0), (0.05, 80.0), (0.4, 3.0)])
def test_1d_potentials_perthame_bouchut(a, lam):
    rho, q, _ = _states(500, 11)
    beta = q / rho
    theta = G * rho - beta * beta / 2.0
    h0, hp, hm = _pot_1d(theta, beta, lam, a)
    p = G * rho * rho / 2.0
    assert np.allclose(h0 + hp + hm, p, rtol=1e-14, atol=0)
    # lam (h+ - h-) cancels O(1) terms: allow lam times a few ulp of them
    assert np.allclose(lam * (hp - hm), p * q / rho, rtol=1e-13, atol=lam * 4e-16 * np.abs(hp).max())


@pytest.mark.parametrize("a,lam", [(0.15, 8.0), (0.0, 8.0), (0.05, 80.0), (0.4, 3.0)])
def test_1d_equilibria_are_potential_derivatives(a, lam):
    rho, q, _ = _states(400, 12)
    p = oracle.params(rho.size, a=a, lam=lam)
    F = oracle.equilibrium_1d(rho, q, p)
    beta = q / rho
    theta = G * rho - beta * beta / 2.0
    eps = 1e-30
    d_theta = [x.imag / eps for x in _pot_1d(theta + 1j * eps, beta, lam, a)]
    d_beta = [x.imag / eps for x in _pot_1d(theta, beta + 1j * eps, lam, a)]
    want = np.array([d_theta[0], d_theta[1], d_theta[2], d_beta[1], d_beta[2]])
    assert np.allclose(d_beta[0], 0.0)  # h_0^* does not depend on beta: no g_0
    np.testing.assert_allclose(F, want, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("a", [0.15, 0.0])
def test_1d_equilibrium_moments_are_physical_fluxes(a):
    lam = 8.0
    rho, q, _ = _states(300, 13)
    F = oracle.equilibrium_1d(rho, q, oracle.params(rho.size, a=a, lam=lam))
    f0, fp, fm, gp, gm = F
    np.testing.assert_allclose(f0 + fp + fm, rho, rtol=1e-14)
    np.testing.assert_allclose(gp + gm, q, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(lam * (fp - fm), q, rtol=1e-12, atol=1e-14)      # J_rho^eq = q
    np.testing.assert_allclose(lam * (gp - gm), q * q / rho + G * rho ** 2 / 2, rtol=1e-13)  # J_q^eq


# --------------------------------------------------------------------- 2D
def _moments_13(F, lam):
    """The 13 moments of section 3, as printed."""
    f0, f1, f2, f3, f4, gx1, gx2, gx3, gx4, gy1, gy2, gy3, gy4 = F
    return dict(
        rho=f0 + f1 + f2 + f3 + f4, Jx=lam * (f1 - f3), Jy=lam * (f2 - f4),
        eps=f1 + f2 + f3 + f4 - 4 * f0, XXr=f1 - f2 + f3 - f4,
        qx=gx1 + gx2 + gx3 + gx4, fxx=lam * (gx1 - gx3), fxy=lam * (gx2 - gx4), XXu=gx1 - gx2 + gx3 - gx4,
        qy=gy1 + gy2 + gy3 + gy4, fyx=lam * (gy1 - gy3), fyy=lam * (gy2 - gy4), XXv=gy1 - gy2 + gy3 - gy4,
    )


@pytest.mark.parametrize("a,lam", [(0.05, 8.0), (0.0, 8.0), (0.05, 80.0), (0.3, 4.0)])
def test_2d_equilibria_match_printed_moment_equilibria(a, lam):
    rho, qx, qy = _states(600, 21)
    p = oracle.params(rho.size, 1, a=a, lam=lam)
    F = oracle.equilibrium_2d(rho, qx, qy, p).reshape(13, -1)
    m = _moments_13(F, lam)
    u, v = qx / rho, qy / rho
    pr = G * rho * rho / 2.0
    rho0_over_c0sq = 1.0 / G  # c0^2 = g rho0
    tol = dict(rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(m["rho"], rho, **tol)
    np.testing.assert_allclose(m["qx"], qx, **tol)
    np.testing.assert_allclose(m["qy"], qy, **tol)
    np.testing.assert_allclose(m["Jx"], qx, **tol)
    np.testing.assert_allclose(m["Jy"], qy, **tol)
    # eps_rho^eq with the factor a on the velocity term (derived from the potentials)
    np.testing.assert_allclose(m["eps"], (1 - 2.5 * a) * rho + 1.25 * a * rho0_over_c0sq * (u * u + v * v), **tol)
    np.testing.assert_allclose(m["XXr"], 0.0, atol=1e-13)
    np.testing.assert_allclose(m["fxx"], rho * u * u + pr, **tol)
    np.testing.assert_allclose(m["fxy"], rho * u * v, **tol)
    np.testing.assert_allclose(m["XXu"], 0.0, atol=1e-13)
    np.testing.assert_allclose(m["fyx"], rho * u * v, **tol)
    np.testing.assert_allclose(m["fyy"], rho * v * v + pr, **tol)
    np.testing.assert_allclose(m["XXv"], 0.0, atol=1e-13)


def test_2d_printed_eps_without_a_is_a_misprint():
    """The printed eps_rho^eq has 5/4 (no a) on the velocity term; the potentials give 5a/4.
    The two agree only at rest, so a moving state tells them apart."""
    a, lam = 0.05, 8.0
    rho, qx, qy = np.array([1.3]), np.array([0.4]), np.array([-0.2])
    F = oracle.equilibrium_2d(rho, qx, qy, oracle.params(1, 1, a=a, lam=lam)).reshape(13, -1)
    eps = _moments_13(F, lam)["eps"][0]
    u2 = (qx[0] ** 2 + qy[0] ** 2) / rho[0] ** 2
    assert abs(eps - ((1 - 2.5 * a) * rho[0] + 1.25 * a * u2)) < 1e-14
    assert abs(eps - ((1 - 2.5 * a) * rho[0] + 1.25 * u2)) > 1e-2


def _pot_2d(theta, u, v, lam, a):
    """Potentials of section 3: h_0^* = (a/2) K theta^2 and the unique solution of the
    constraints (3-st-venant-contraintes-2) and the split (3-st-venant-enplus)."""
    K = 1.0 / (2.0 * G)
    p = K * (theta + (u * u + v * v) / 2.0) ** 2
    h0 = a / 2.0 * K * theta * theta
    h1 = (p - h0) / 4.0 + p * u / (2.0 * lam)
    h3 = (p - h0) / 4.0 - p * u / (2.0 * lam)
    h2 = (p - h0) / 4.0 + p * v / (2.0 * lam)
    h4 = (p - h0) / 4.0 - p * v / (2.0 * lam)
    return p, (h0, h1, h2, h3, h4)


def test_2d_potentials_satisfy_constraints():
    a, lam = 0.05, 8.0
    rho, qx, qy = _states(300, 22)
    u, v = qx / rho, qy / rho
    theta = G * rho - (u * u + v * v) / 2.0
    p, (h0, h1, h2, h3, h4) = _pot_2d(theta, u, v, lam, a)
    np.testing.assert_allclose(p, G * rho * rho / 2.0, rtol=1e-14)
    np.testing.assert_allclose(h0 + h1 + h2 + h3 + h4, p, rtol=1e-14)
    np.testing.assert_allclose(lam * (h1 - h3), p * u, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(lam * (h2 - h4), p * v, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(h1 + h3, (p - h0) / 2.0, rtol=1e-14)
    np.testing.assert_allclose(h2 + h4, (p - h0) / 2.0, rtol=1e-14)


@pytest.mark.parametrize("a,lam", [(0.05, 8.0), (0.0, 8.0), (0.05, 80.0)])
def test_2d_equilibria_are_potential_derivatives(a, lam):
    rho, qx, qy = _states(300, 23)
    F = oracle.equilibrium_2d(rho, qx, qy, oracle.params(rho.size, 1, a=a, lam=lam)).reshape(13, -1)
    u, v = qx / rho, qy / rho
    theta = G * rho - (u * u + v * v) / 2.0
    eps = 1e-30
    dt = [x.imag / eps for x in _pot_2d(theta + 1j * eps, u, v, lam, a)[1]]
    du = [x.imag / eps for x in _pot_2d(theta, u + 1j * eps, v, lam, a)[1]]
    dv = [x.imag / eps for x in _pot_2d(theta, u, v + 1j * eps, lam, a)[1]]
    assert np.allclose(du[0], 0) and np.allclose(dv[0], 0)  # no gx0, gy0
    want = np.array(dt + du[1:] + dv[1:])
    np.testing.assert_allclose(F, want, rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------- collision
def _conserved_2d(F):
    return F[0:5].sum(0), F[5:9].sum(0), F[9:13].sum(0)


@pytest.mark.parametrize("s", [1.8, 1.0, 0.5, 1.99])
def test_2d_collision_conserves_moments(s):
    F = inputs.random_populations(13, 6, 9, seed=31)
    p = oracle.params(9, 6, s=s)
    Fs = oracle.collide_2d(F, p)
    for before, after in zip(_conserved_2d(F), _conserved_2d(Fs)):
        np.testing.assert_allclose(after, before, rtol=1e-14, atol=1e-15)


def test_2d_collision_limits():
    F = inputs.random_populations(13, 4, 5, seed=32)
    assert np.array_equal(oracle.collide_2d(F, oracle.params(5, 4, s=0.0)), F)
    rho, qx, qy = _conserved_2d(F)
    feq = oracle.equilibrium_2d(rho, qx, qy, oracle.params(5, 4))
    np.testing.assert_allclose(oracle.collide_2d(F, oracle.params(5, 4, s=1.0)), feq, rtol=0, atol=1e-15)
    # an equilibrium is a fixed point of the collision
    np.testing.assert_allclose(oracle.collide_2d(feq, oracle.params(5, 4, s=1.8)), feq, rtol=0, atol=1e-15)


def test_1d_collision_conserves_and_limits():
    F = inputs.random_populations(5, 1, 40, seed=33).reshape(5, 40)
    Fs = oracle.collide_1d(F, oracle.params(40, a=0.15, s=1.8))
    np.testing.assert_allclose(Fs[0:3].sum(0), F[0:3].sum(0), rtol=1e-14)
    np.testing.assert_allclose(Fs[3:5].sum(0), F[3:5].sum(0), rtol=1e-13, atol=1e-15)
    assert np.array_equal(oracle.collide_1d(F, oracle.params(40, a=0.15, s=0.0)), F)
    feq = oracle.equilibrium_1d(F[0:3].sum(0), F[3:5].sum(0), oracle.params(40, a=0.15))
    np.testing.assert_allclose(oracle.collide_1d(F, oracle.params(40, a=0.15, s=1.0)), feq, atol=1e-15)


def test_2d_mrt_equal_rates_is_bgk():
    F = inputs.random_populations(13, 5, 6, seed=34)
    bgk = oracle.collide_2d(F, oracle.params(6, 5, s=1.7))
    mrt = oracle.collide_2d(F, oracle.params(6, 5, s=1.7, s_moments=[1.7] * 13))
    np.testing.assert_allclose(mrt, bgk, rtol=1e-13, atol=1e-14)


def test_2d_mrt_relaxes_each_printed_moment_at_its_rate():
    lam = 8.0
    F = inputs.random_populations(13, 3, 4, seed=35)
    rates = [0.0, 1.1, 1.2, 1.3, 1.4, 0.0, 1.5, 1.6, 1.7, 0.0, 1.8, 1.9, 0.9]
    out = oracle.collide_2d(F, oracle.params(4, 3, lam=lam, s_moments=rates))
    rho, qx, qy = _conserved_2d(F)
    feq = oracle.equilibrium_2d(rho, qx, qy, oracle.params(4, 3, lam=lam))
    m, meq, mo = _moments_13(F, lam), _moments_13(feq, lam), _moments_13(out, lam)
    for k, name in enumerate(m):
        want = m[name] + rates[k] * (meq[name] - m[name])
        np.testing.assert_allclose(mo[name], want, rtol=1e-12, atol=1e-13, err_msg=name)


def test_1d_mrt_relaxes_each_printed_moment_at_its_rate():
    lam, a = 8.0, 0.15
    F = inputs.random_populations(5, 1, 30, seed=36).reshape(5, 30)
    rates = [0.0, 1.3, 1.6, 0.0, 1.9]
    out = oracle.collide_1d(F, oracle.params(30, lam=lam, a=a, s_moments=rates))
    feq = oracle.equilibrium_1d(F[0:3].sum(0), F[3:5].sum(0), oracle.params(30, lam=lam, a=a))

    def mom(f):  # rho, J_rho, eps_rho, q, J_q of section 2, as printed
        return [f[0] + f[1] + f[2], lam * (f[1] - f[2]), lam * lam * (f[1] + f[2] - 2 * f[0]),
                f[3] + f[4], lam * (f[3] - f[4])]

    for k, (mk, mek, mok) in enumerate(zip(mom(F), mom(feq), mom(out))):
        np.testing.assert_allclose(mok, mk + rates[k] * (mek - mk), rtol=1e-12, atol=1e-12)
