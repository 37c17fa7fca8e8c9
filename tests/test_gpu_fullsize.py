"""Parity at the benchmark size: the 4096 x 4096 two-phase workload, in the
configuration bench.py times (walls in y, F_eps = 0, tau = 1, G = 1e-6,
16-byte vector path), against the full-lattice FP64 oracle (OpenMP build)
after a few steps; every node is compared.  Plus a very wide ragged lattice
(65540 x 4)."""

import numpy as np
import pytest

import media

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.fixture(scope="module")
def pkg():
    from paper_1601_00704_gb300 import build
    build.build()
    import paper_1601_00704_gb300 as p
    return p


@pytest.fixture(scope="module")
def full(orc):
    n = 4096
    eps, K, _ = media.two_phase_medium(n, n, seed=0)
    o = orc.Oracle(n, n, tau=1.0, threads=16)
    o.set_medium(eps, K)
    o.set_force(1e-6)
    o.step(6)
    return eps, K, o


@pytest.mark.parametrize("storage,ulp", [("f32", 2.0 ** -23), ("bf16", 2.0 ** -7), ("f16", 2.0 ** -10)])
def test_benchmark_size_matches_oracle(pkg, full, storage, ulp):
    eps, K, o = full
    n = eps.shape[0]
    s = pkg.Solver(n, n, tau=1.0, storage=storage)
    s.set_medium(eps, K)
    s.set_force(1e-6)
    s.step(6)
    f = s.distributions()
    g_orc = o.f - W[:, None, None]
    gmax = np.abs(g_orc).max()
    err = np.abs(f - o.f).max()
    print(f"{storage}: max |df| {err:.3e} (max |g| {gmax:.3e})")
    assert err <= 2 * 6 * ulp * gmax + 1e-15
    ux, uy = s.velocity()
    assert np.abs(ux - o.ux).max() <= 2 * 6 * ulp * gmax * 10
    assert s.mean_velocity()[0] == pytest.approx(o.mean_u[0], rel=max(100 * ulp, 1e-6))


def test_very_wide_ragged_lattice(pkg, orc):
    """65540 nodes per row (128 blocks + a ragged tail of one thread)."""
    nx, ny = 65540, 4
    eps, K = media.random_medium(nx, ny, seed=77)
    s = pkg.Solver(nx, ny, tau=0.8, storage="f32")
    s.set_medium(eps, K)
    s.set_force(3e-4, -1e-4)
    s.step(3)
    o = orc.Oracle(nx, ny, tau=0.8)
    o.set_medium(eps, K)
    o.set_force(3e-4, -1e-4)
    o.step(3)
    gmax = np.abs(o.f - W[:, None, None]).max()
    np.testing.assert_allclose(s.distributions(), o.f, rtol=0, atol=1e-6 * 3 * gmax)
