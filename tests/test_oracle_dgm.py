"""Pins of the DGM/GMS apparent-permeability oracle (Sec. 2.1, Eqs. 3-4,
18-19, 38) against structural properties the formulas must have."""

import math

import numpy as np
import pytest

# Table "Input parameters of IOM": 22/20 MPa, eta 18.231e-6 Pa s, tortuosity
# 2, porosity 0.04; methane at 350 K (the temperature the tables omit).
P_MEAN, ETA, TORT, EPS, T = 21e6, 18.231e-6, 2.0, 0.04, 350.0
# OM surface-diffusion inputs of Sec. 3.1.2: D_s 5e-7 m^2/s, q 4000 mol/m^3,
# b 0.25 MPa^-1
DS, QSAT, B = 5e-7, 4000.0, 0.25e-6


def test_k0_kc_relation(orc):
    """Eq. 4: K_c = (8/d_p) K0 = (eps/tau)(d_p/4), hence K0 = eps d_p^2/(32 tau);
    K0 is the capillary-bundle permeability, quadratic in the radius."""
    for r in (1e-9, 5e-9, 2e-8):
        Kc, K0 = orc.dgm_kc_k0(r, EPS, TORT)
        d = 2 * r
        assert Kc == pytest.approx(8 / d * K0, rel=1e-14)
        assert Kc == pytest.approx(EPS / TORT * d / 4, rel=1e-14)
    _, a = orc.dgm_kc_k0(1e-9, EPS, TORT)
    _, b = orc.dgm_kc_k0(3e-9, EPS, TORT)
    assert b / a == pytest.approx(9.0, rel=1e-13)


def test_knudsen_kinetic_theory(orc):
    """Eq. 3 is (4/3) K_c times the mean molecular speed sqrt(8RT/(pi M));
    for methane at 350 K that speed is ~680 m/s (kinetic theory)."""
    vbar = orc.knudsen_diffusivity(0.75, T)
    assert 670 < vbar < 690
    assert orc.knudsen_diffusivity(1.5, 4 * T) == pytest.approx(4 * vbar, rel=1e-14)


def test_eq19_reduces_to_eq18_without_surface_diffusion(orc):
    for r in (1e-9, 4e-9, 5e-8):
        iom = orc.kapp(r, P_MEAN, T, ETA, EPS, TORT, False)
        assert orc.kapp(r, P_MEAN, T, ETA, EPS, TORT, True, QSAT, B, 0.0) == pytest.approx(iom, rel=1e-14)
        assert orc.kapp(r, P_MEAN, T, ETA, EPS, TORT, True, 0.0, B, DS) == pytest.approx(iom, rel=1e-14)


def test_linear_in_qsat(orc):
    """Sec. 3.1.2 (Langmuir study): K_app of OM is linear in q_sat."""
    r = 11e-9
    k = [orc.kapp(r, P_MEAN, T, ETA, EPS, TORT, True, q, B, DS) for q in (0, 2000, 4000, 8000)]
    assert k[2] - k[0] == pytest.approx(2 * (k[1] - k[0]), rel=1e-10)
    assert k[3] - k[0] == pytest.approx(4 * (k[1] - k[0]), rel=1e-10)


def test_pressure_dependence(orc):
    """Sec. 3.1.1: K0 does not depend on P while the Knudsen part falls as
    1/P, so K_app -> K0 as P -> infinity; the surface part of OM falls with P."""
    r = 2e-9
    _, K0 = orc.dgm_kc_k0(r, EPS, TORT)
    k1 = orc.kapp(r, 1e6, T, ETA, EPS, TORT, False) - K0
    k4 = orc.kapp(r, 4e6, T, ETA, EPS, TORT, False) - K0
    assert k1 == pytest.approx(4 * k4, rel=1e-12)
    assert orc.kapp(r, 1e15, T, ETA, EPS, TORT, False) == pytest.approx(K0, rel=1e-7)
    s = [orc.kapp(r, P, T, ETA, EPS, TORT, True, QSAT, B, DS) - orc.kapp(r, P, T, ETA, EPS, TORT, False)
         for P in (1e6, 5e6, 2e7)]
    assert s[0] > s[1] > s[2] > 0


def test_radius_scaling(orc):
    """Doubling the radius multiplies K0 by 4 and the Knudsen part by 2 and
    leaves the surface-diffusion part unchanged."""
    r = 3e-9
    _, K0 = orc.dgm_kc_k0(r, EPS, TORT)
    kn = orc.kapp(r, P_MEAN, T, ETA, EPS, TORT, False) - K0
    sf = orc.kapp(r, P_MEAN, T, ETA, EPS, TORT, True, QSAT, B, DS) - kn - K0
    k2 = orc.kapp(2 * r, P_MEAN, T, ETA, EPS, TORT, True, QSAT, B, DS)
    assert k2 == pytest.approx(4 * K0 + 2 * kn + sf, rel=1e-12)


def test_large_pores_reach_k0(orc):
    """Sec. 3.1.1: near 100 nm and beyond, Knudsen diffusion no longer matters
    (K_app ~ K0); at 10 microns the excess is below 1 percent."""
    _, K0 = orc.dgm_kc_k0(1e-5, EPS, TORT)
    assert orc.kapp(1e-5, P_MEAN, T, ETA, EPS, TORT, False) / K0 - 1 < 1e-2


def test_surface_diffusion_dominates_nanopores(orc):
    """Sec. 3.1.2: with D_s 5e-7, q 4000 mol/m^3, b 0.25 MPa^-1 and the IOM
    table's other inputs, K_app/K0 of OM exceeds 10 for r < 2 nm."""
    for r in (1.0e-9, 1.5e-9, 1.99e-9):
        _, K0 = orc.dgm_kc_k0(r, EPS, TORT)
        assert orc.kapp(r, P_MEAN, T, ETA, EPS, TORT, True, QSAT, B, DS) / K0 > 10


def test_langmuir_volume_conversion(orc):
    """Eq. 38 is linear in q_sat,b and rho_b and inversely proportional to
    (1 - eps) TOC and to M_CH4.  (The paper's 1000-8000 mol/m^3 band rests on
    Langmuir volumes and TOC values shown only in a figure, so it is not a
    pin here.)"""
    q = orc.qsat_from_langmuir_volume(0.004, 1.65e3, 0.2, 0.5, 0.717)
    assert orc.qsat_from_langmuir_volume(0.008, 1.65e3, 0.2, 0.5, 0.717) == pytest.approx(2 * q, rel=1e-14)
    assert orc.qsat_from_langmuir_volume(0.004, 3.3e3, 0.2, 0.5, 0.717) == pytest.approx(2 * q, rel=1e-14)
    assert orc.qsat_from_langmuir_volume(0.004, 1.65e3, 0.6, 0.5, 0.717) == pytest.approx(2 * q, rel=1e-14)
    assert orc.qsat_from_langmuir_volume(0.004, 1.65e3, 0.2, 0.25, 0.717) == pytest.approx(2 * q, rel=1e-14)
    assert orc.qsat_from_langmuir_volume(0.004, 1.65e3, 0.2, 0.5, 0.717, 0.00802) == pytest.approx(2 * q, rel=1e-14)


def test_field_matches_pointwise(orc):
    rng = np.random.default_rng(0)
    r = rng.lognormal(math.log(5e-9), 0.5, 100)
    org = rng.random(100) < 0.3
    eps = np.where(org, 0.04, 0.02)
    K = orc.kapp_field(r, org, eps, 5e6, T, ETA, TORT, QSAT, B, DS, 7.8125e-9)
    for i in range(0, 100, 7):
        want = orc.kapp(r[i], 5e6, T, ETA, eps[i], TORT, bool(org[i]), QSAT, B, DS) / 7.8125e-9 ** 2
        assert K[i] == pytest.approx(want, rel=1e-15)
