"""Pins of the oracle's per-node pieces against what the mathematics fixes.

Each identity below follows from the D2Q9 lattice (c_s^2 = 1/3) and the
moment conditions that the equilibrium (Eq. 30) and the forcing term
(Eq. 31) are built to satisfy; none re-types the oracle's formulas.
"""

import math

import numpy as np
import pytest

# D2Q9 directions and weights, written from the lattice definition.
E = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1),
              (1, 1), (-1, 1), (-1, -1), (1, -1)], dtype=float)
CS2 = 1.0 / 3.0

rng = np.random.default_rng(1234)
CASES = [(1.0 + 0.1 * rng.standard_normal(), 0.05 * rng.standard_normal(2),
          rng.uniform(0.05, 1.0)) for _ in range(20)]


def moments(f):
    m0 = f.sum()
    m1 = E.T @ f
    m2 = np.einsum("i,ia,ib->ab", f, E, E)
    return m0, m1, m2


@pytest.mark.parametrize("rho,u,eps", CASES)
def test_equilibrium_moments(orc, rho, u, eps):
    """Eq. 30: zeroth, first and second moments of the eps-equilibrium are
    rho, rho*u and rho*c_s^2*I + rho*u u/eps (the porous-medium momentum
    flux of the generalized NS equation, Eq. 26)."""
    feq = orc.equilibrium(rho, u[0], u[1], eps)
    m0, m1, m2 = moments(feq)
    assert m0 == pytest.approx(rho, rel=1e-15, abs=1e-15)
    np.testing.assert_allclose(m1, rho * u, rtol=1e-13, atol=1e-17)
    want = rho * CS2 * np.eye(2) + rho * np.outer(u, u) / eps
    np.testing.assert_allclose(m2, want, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("rho,u,eps", CASES)
def test_forcing_moments(orc, rho, u, eps):
    """Eq. 31 (reading: -(3/eps) u.F): sum F_i = 0 (no mass source),
    sum F_i e = rho(1-1/2tau)F, sum F_i e e = rho(1-1/2tau)(uF+Fu)/eps."""
    tau = 0.6 + rng.uniform(0, 1.5)
    F = 1e-3 * rng.standard_normal(2)
    Fi = orc.forcing(rho, u[0], u[1], F[0], F[1], eps, tau)
    m0, m1, m2 = moments(Fi)
    a = rho * (1.0 - 0.5 / tau)
    scale = a * np.abs(F).max()
    assert abs(m0) < 1e-15 * max(scale, 1e-30) + 1e-19
    np.testing.assert_allclose(m1, a * F, rtol=1e-13, atol=1e-19)
    want = a * (np.outer(u, F) + np.outer(F, u)) / eps
    np.testing.assert_allclose(m2, want, rtol=1e-12, atol=1e-19)


def test_literal_forcing_creates_mass(orc):
    """The printed Eq. 31 (last term without 1/eps) has a mass source
    3 rho (1-1/2tau)(1/eps - 1) u.F, which is why the default reading adds
    the 1/eps.  At eps = 1 the two readings coincide."""
    rho, ux, uy, Fx, Fy, eps, tau = 1.01, 0.03, -0.02, 2e-3, 5e-4, 0.4, 0.9
    lit = orc.forcing(rho, ux, uy, Fx, Fy, eps, tau, literal=True)
    src = 3 * rho * (1 - 0.5 / tau) * (1 / eps - 1) * (ux * Fx + uy * Fy)
    assert lit.sum() == pytest.approx(src, rel=1e-12)
    a = orc.forcing(rho, ux, uy, Fx, Fy, 1.0, tau, literal=True)
    b = orc.forcing(rho, ux, uy, Fx, Fy, 1.0, tau, literal=False)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-18)


@pytest.mark.parametrize("seed", range(12))
def test_velocity_solves_eq33(orc, seed):
    """Eq. 34 is the explicit root of Eq. 33 with F from Eq. 27: the returned
    u must satisfy rho*u = sum f e + rho*F(u)/2, and the Darcy/Forchheimer
    coefficients must match Eqs. 36-37's definitions."""
    r = np.random.default_rng(seed)
    rho = 1 + 0.05 * r.standard_normal()
    m = 1e-2 * r.standard_normal(2)
    eps = r.uniform(0.05, 1.0)
    K = 10 ** r.uniform(-5, 2)
    feps = [0.0, 0.7, -1.0][seed % 3]
    fe = orc.feps(feps, eps)
    nu = (r.uniform(0.55, 2.0) - 0.5) / 3
    g = 1e-3 * r.standard_normal(2)
    ux, uy = orc.velocity(rho, m[0], m[1], eps, K, fe, nu, g[0], g[1])
    Fx, Fy = orc.body_force(ux, uy, eps, K, fe, nu, g[0], g[1])
    lhs = rho * np.array([ux, uy])
    rhs = m + 0.5 * rho * np.array([Fx, Fy])
    np.testing.assert_allclose(lhs, rhs, rtol=1e-11,
                               atol=1e-15 * np.abs(m).max())
    # Darcy drag coefficient: eps*nu/K = 4*c0 - 2; Forchheimer: eps*F/sqrt(K) = 2*c1
    c0, c1 = orc.c0_c1(eps, K, fe, nu)
    assert 4 * c0 - 2 == pytest.approx(eps * nu / K, rel=1e-9)
    assert 2 * c1 == pytest.approx(eps * fe / math.sqrt(K), rel=1e-12, abs=1e-300)


def test_clear_fluid_limits(orc):
    """K = +inf: no drag, c0 = 1/2, c1 = 0, u = v (standard Guo velocity)."""
    c0, c1 = orc.c0_c1(0.3, math.inf, 0.5, 1 / 6)
    assert c0 == 0.5 and c1 == 0.0
    ux, uy = orc.velocity(1.2, 0.012, -0.006, 1.0, math.inf, 0.0, 1 / 6, 1e-3, 0)
    assert ux == pytest.approx(0.012 / 1.2 + 0.5e-3, rel=1e-15)
    assert uy == pytest.approx(-0.006 / 1.2, rel=1e-15)


def test_ergun_reading(orc):
    """F_eps < 0 selects Ergun's 1.75/sqrt(150 eps^3); 0 gives none; >0 is
    taken as given."""
    for eps in (0.1, 0.4, 1.0):
        assert orc.feps(-1.0, eps) == pytest.approx(
            1.75 / math.sqrt(150 * eps ** 3), rel=1e-15)
    assert orc.feps(0.0, 0.3) == 0.0
    assert orc.feps(0.25, 0.3) == 0.25


def test_permeability_is_darcy(orc):
    """K_app = nu <u_x> / G_x with nu = (tau - 1/2)/3."""
    assert orc.permeability(1.0, 6e-4, 1e-6) == pytest.approx(100.0, rel=1e-14)
