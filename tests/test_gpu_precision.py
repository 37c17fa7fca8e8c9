"""Reduced-precision storage (FP16 / BF16 deviations) against the FP64 oracle.

Tolerances:
* a few steps on random media: each stored deviation carries one rounding of
  at most 1 ulp (stochastic rounding) of the format -- 2^-10 relative for
  FP16, 2^-7 for BF16 -- so after n steps |df| <= 2 n ulp max|g|;
* the 128x128 two-phase parity workload after 3000 steps: the north-star
  target, |K_app / K_app(oracle) - 1| <= 1e-3, for both formats and both the
  narrow (config 0) and the wide K range [1e-6, 1e-2] (config 2 media).
"""

import math

import numpy as np
import pytest

import media

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
ULP = {"f16": 2.0 ** -10, "bf16": 2.0 ** -7}


@pytest.fixture(scope="module")
def pkg():
    from paper_1601_00704_gb300 import build
    build.build()
    import paper_1601_00704_gb300 as p
    return p


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("nx,ny,walls", [(64, 12, True), (37, 9, False), (516, 3, True)])
def test_steps_match_oracle_16bit(pkg, orc, storage, nx, ny, walls):
    eps, K = media.random_medium(nx, ny, seed=nx + 7 * ny)
    s = pkg.Solver(nx, ny, tau=0.8, storage=storage, walls=walls)
    s.set_medium(eps, K)
    s.set_force(3e-4, -1e-4)
    o = orc.Oracle(nx, ny, tau=0.8, periodic_y=not walls)
    o.set_medium(eps, K)
    o.set_force(3e-4, -1e-4)
    for n in (1, 4):
        s.step(n)
        o.step(n)
        gmax = np.abs(o.f - W[:, None, None]).max()
        np.testing.assert_allclose(s.distributions(), o.f, rtol=0,
                                   atol=2 * o.steps * ULP[storage] * gmax)


def medium(kind):
    if kind == "c0":
        eps, K, _ = media.two_phase_medium(128, 128, seed=0)
    else:  # config-2 K spread
        eps, K, _ = media.two_phase_medium(128, 128, seed=0, k_iom=(1e-6, 1e-2),
                                           k_om=(1e-6, 1e-2))
    return eps, K


@pytest.fixture(scope="module")
def oracle_runs(orc):
    out = {}
    for kind in ("c0", "c2"):
        eps, K = medium(kind)
        o = orc.Oracle(128, 128, threads=8)
        o.set_medium(eps, K)
        o.set_force(1e-6)
        o.step(3000)
        out[kind] = (eps, K, o)
    return out


@pytest.mark.parametrize("kind", ["c0", "c2"])
@pytest.mark.parametrize("storage", ["f16", "bf16", "f32"])
def test_kapp_reduced_precision_128(pkg, oracle_runs, kind, storage):
    eps, K, o = oracle_runs[kind]
    s = pkg.Solver(128, 128, storage=storage)
    s.set_medium(eps, K)
    s.set_force(1e-6)
    s.step(3000)
    ux, _ = s.velocity()
    rk = s.permeability() / o.permeability() - 1
    ru = np.linalg.norm(ux - o.ux) / np.linalg.norm(o.ux)
    print(f"{kind} {storage}: K_app rel {rk:+.3e}, u_x rel L2 {ru:.3e}")
    assert abs(rk) <= 1e-3


def test_nearest_rounding_stagnates(pkg, oracle_runs):
    """Round-to-nearest FP16 loses the slow pressure mode (its K_app error is
    several times the stochastic-rounding error)."""
    eps, K, o = oracle_runs["c0"]
    err = {}
    for flag, name in ((0, "sr"), (pkg.NEAREST16, "rn")):
        s = pkg.Solver(128, 128, storage="f16", flags=flag)
        s.set_medium(eps, K)
        s.set_force(1e-6)
        s.step(3000)
        err[name] = abs(s.permeability() / o.permeability() - 1)
    print(f"FP16 K_app rel error: stochastic {err['sr']:.2e}, nearest {err['rn']:.2e}")
    assert err["sr"] < err["rn"]


def test_stochastic_rounding_reproducible(pkg):
    eps, K, _ = media.two_phase_medium(96, 64, seed=4)
    runs = []
    for _ in range(2):
        s = pkg.Solver(96, 64, storage="bf16")
        s.set_medium(eps, K)
        s.set_force(1e-6)
        s.step(200)
        runs.append(s.distributions())
    assert np.array_equal(runs[0], runs[1])


def test_fp16_scale_adapts(pkg, orc):
    """A warm start with O(0.05) velocities and density deviations sets the
    FP16 scale from the initial state; the run then decays towards the Darcy
    state over ~4 decades without overflow or loss against FP32."""
    nx, ny = 64, 32
    eps, K = media.uniform_medium(nx, ny, 0.5, 1e-2)
    rho, ux, uy = media.random_state(nx, ny, seed=3, amp=2e-2, u_amp=0.05)
    res = {}
    for storage in ("f32", "f16"):
        s = pkg.Solver(nx, ny, storage=storage)
        s.set_medium(eps, K)
        s.set_force(1e-6)
        s.init_equilibrium(rho, ux, uy)
        s.step(4000, check_every=100)
        res[storage] = s.distributions() - W[:, None, None]
    gmax = np.abs(res["f32"]).max()
    assert np.isfinite(res["f16"]).all()
    np.testing.assert_allclose(res["f16"], res["f32"], rtol=0, atol=0.05 * gmax)
