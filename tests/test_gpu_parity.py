"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances, derived from the arithmetic:
* FP64 storage (deviations, FP64 collide): the oracle itself stores absolute
  f in FP64, so each f is resolved to ~1e-17; after n steps the two agree to
  ~n * 1e-16 on f.  Bound: |df| <= 1e-14.
* FP32 storage: every stored deviation is rounded to ~6e-8 relative per
  step; after n steps |dg| <= ~n * 6e-8 * max|g|.  Bound: 1e-6 * n * max|g|.
* Converged 128x128 two-phase medium (the parity workload): relative L2 of
  the velocity field <= 1e-5 and relative K_app <= 1e-4 for FP32; 1e-7 /
  1e-7 for FP64 storage (limited by the oracle's absolute-f round-off).
"""

import math

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
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return p


def pair(pkg, orc, eps, K, g, *, tau=1.0, walls=True, storage="f32", feps=0.0):
    ny, nx = eps.shape
    s = pkg.Solver(nx, ny, tau=tau, storage=storage, walls=walls)
    s.set_medium(eps, K, feps)
    s.set_force(*g)
    o = orc.Oracle(nx, ny, tau=tau, periodic_y=not walls)
    o.set_medium(eps, K, feps)
    o.set_force(*g)
    return s, o


SHAPES = [(16, 16), (17, 9), (64, 6), (6, 5), (2, 2), (516, 3), (1030, 4)]


@pytest.mark.parametrize("storage,tol_f", [("f64", 1e-14), ("f32", None)])
@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("walls", [True, False])
@pytest.mark.parametrize("feps", [0.0, -1.0, 2.0])
def test_steps_match_oracle(pkg, orc, storage, tol_f, nx, ny, walls, feps):
    """1, 2 and 10 steps on random media with large velocities, every shape
    class: vector path (nx multiple of the vector width), scalar path,
    ragged last block (nx = 4*128 + 4, 1030), minimal 2x2 lattice."""
    eps, K = media.random_medium(nx, ny, seed=nx * 131 + ny)
    s, o = pair(pkg, orc, eps, K, (3e-4, -1e-4), tau=0.8, walls=walls,
                storage=storage, feps=feps)
    for n in (1, 1, 8):
        s.step(n)
        o.step(n)
        f = s.distributions()
        gmax = np.abs(o.f - W[:, None, None]).max()
        tol = tol_f if tol_f is not None else 1e-6 * o.steps * gmax
        np.testing.assert_allclose(f, o.f, rtol=0, atol=tol)
        ux, uy = s.velocity()
        umax = np.abs(o.ux).max()
        utol = (1e-12 if storage == "f64" else 2e-5 * o.steps) * umax
        np.testing.assert_allclose(ux, o.ux, rtol=0, atol=utol)
        np.testing.assert_allclose(uy, o.uy, rtol=0, atol=utol)
        mu = s.mean_velocity()
        np.testing.assert_allclose(mu, o.mean_u, rtol=0, atol=utol)


def test_warm_start_equilibrium(pkg, orc):
    """init_equilibrium(rho, u) sets f = f_eq(rho, u; eps) (Eq. 30): FP64
    storage to round-off, FP32 to 2 ulps of the largest stored deviation."""
    nx, ny = 24, 20
    eps, K = media.random_medium(nx, ny, seed=9)
    rho, ux, uy = media.random_state(nx, ny, seed=10)
    for storage in ("f64", "f32"):
        s, o = pair(pkg, orc, eps, K, (0.0, 0.0), storage=storage)
        s.init_equilibrium(rho, ux, uy)
        o.init_equilibrium(rho, ux, uy)
        gmax = np.abs(o.f - W[:, None, None]).max()
        tol = 1e-15 if storage == "f64" else 2.4e-7 * gmax
        np.testing.assert_allclose(s.distributions(), o.f, rtol=0, atol=tol)
        s.step(5)
        o.step(5)
        np.testing.assert_allclose(s.distributions(), o.f, rtol=0, atol=6 * tol)


_CONFIG0 = {}


def config0(orc, seed):
    """The 128x128 parity workload: two-phase OM/IOM medium (OM fraction 0.2,
    correlation length 8), G = 1e-6 along x, tau = 1, walls in y, run to a
    relative change of mean u_x below 1e-10 per 100 steps or 10000 steps."""
    if seed not in _CONFIG0:
        eps, K, _ = media.two_phase_medium(128, 128, om_fraction=0.2, corr_len=8, seed=seed)
        o = orc.Oracle(128, 128, tau=1.0, threads=8)
        o.set_medium(eps, K)
        o.set_force(1e-6, 0.0)
        done, conv = o.step(10000, tol=1e-10, check_every=100)
        _CONFIG0[seed] = (eps, K, o, done, conv)
    return _CONFIG0[seed]


@pytest.mark.parametrize("storage,seed,tol_u,tol_k", [("f64", 0, 1e-7, 1e-7),
                                                      ("f32", 0, 1e-5, 1e-4),
                                                      ("f32", 1, 1e-5, 1e-4),
                                                      ("f32", 2, 1e-5, 1e-4)])
def test_converged_128_two_phase(pkg, orc, storage, seed, tol_u, tol_k):
    eps, K, o, done, conv = config0(orc, seed)
    s = pkg.Solver(128, 128, tau=1.0, storage=storage)
    s.set_medium(eps, K)
    s.set_force(1e-6, 0.0)
    sd, sc = s.step(10000, tol=1e-10, check_every=100)
    ux, uy = s.velocity()
    # compare at the oracle's converged state: run the GPU to the same step
    if sd < done:
        s.step(done - sd)
        ux, uy = s.velocity()
    rel_u = math.hypot(np.linalg.norm(ux - o.ux), np.linalg.norm(uy - o.uy)) / \
        math.hypot(np.linalg.norm(o.ux), np.linalg.norm(o.uy))
    rel_k = abs(s.permeability() / o.permeability() - 1)
    print(f"{storage} seed {seed}: oracle steps {done} conv {conv}; gpu steps {sd} conv {sc}; "
          f"velocity rel L2 {rel_u:.3e}; K_app rel {rel_k:.3e}")
    assert rel_u <= tol_u
    assert rel_k <= tol_k


# -- closed forms through the library ------------------------------------

@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_darcy_fixed_point(pkg, storage):
    eps, K = media.uniform_medium(64, 8, 0.3, 2e-3)
    s = pkg.Solver(64, 8, tau=1.0, storage=storage, walls=False)
    s.set_medium(eps, K)
    s.set_force(1e-6, 0.0)
    s.step(20000, tol=1e-13, check_every=50)
    assert s.permeability() == pytest.approx(2e-3, rel=1e-6 if storage == "f32" else 1e-9)


def test_poiseuille_magic_tau(pkg):
    tau = 0.5 + math.sqrt(3) / 4
    ny = 32
    eps, K = media.uniform_medium(8, ny, 1.0, math.inf)
    s = pkg.Solver(8, ny, tau=tau, storage="f64")
    s.set_medium(eps, K)
    s.set_force(1e-6, 0.0)
    s.step(500000, tol=1e-14, check_every=100)
    ux, _ = s.velocity()
    nu = (tau - 0.5) / 3
    y = np.arange(ny)
    prof = 1e-6 / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    np.testing.assert_allclose(ux, np.broadcast_to(prof[:, None], ux.shape), rtol=1e-9)
    assert s.permeability() == pytest.approx((ny ** 2 + 0.5) / 12, rel=1e-9)


def test_mean_velocity_matches_fsum(pkg):
    eps, K, _ = media.two_phase_medium(256, 96, seed=3)
    s = pkg.Solver(256, 96)
    s.set_medium(eps, K)
    s.set_force(1e-6)
    s.step(300)
    ux, uy = s.velocity()
    mu = s.mean_velocity()
    assert mu[0] == pytest.approx(math.fsum(ux.ravel()) / ux.size, rel=1e-12)
    assert mu[1] == pytest.approx(math.fsum(uy.ravel()) / uy.size, abs=1e-12 * abs(mu[0]))


def test_mass_drift_fp32(pkg):
    """Mass is conserved in arithmetic; FP32 deviation storage keeps the
    total within round-off of the deviations (stated bound 1e-12 relative
    over 2000 steps)."""
    eps, K, _ = media.two_phase_medium(128, 128, seed=5)
    s = pkg.Solver(128, 128)
    s.set_medium(eps, K)
    s.set_force(1e-6)
    s.step(2000)
    f = s.distributions()
    assert abs(f.sum() / 128 ** 2 - 1) < 1e-12


def test_device_arrays_and_stream(pkg, orc):
    """Device (torch CUDA) inputs/outputs and a user stream give the same
    result as host arrays."""
    import torch
    eps, K = media.random_medium(32, 16, seed=21)
    st = torch.cuda.Stream()
    a = pkg.Solver(32, 16, tau=0.9, stream=st)
    a.set_medium(torch.from_numpy(eps).cuda(), torch.from_numpy(K).cuda())
    a.set_force(1e-4)
    a.step(20)
    ux = torch.empty((16, 32), dtype=torch.float64, device="cuda")
    uy = torch.empty_like(ux)
    a.velocity(ux, uy)
    st.synchronize()
    b = pkg.Solver(32, 16, tau=0.9)
    b.set_medium(eps, K)
    b.set_force(1e-4)
    b.step(20)
    bx, _ = b.velocity()
    assert np.array_equal(ux.cpu().numpy(), bx)


def test_errors(pkg):
    with pytest.raises(pkg.GLBMError) as e:
        pkg.Solver(1, 4)
    assert e.value.name == "GLBM_EINVAL"
    with pytest.raises(pkg.GLBMError):
        pkg.Solver(4, 4, tau=0.5)
    s = pkg.Solver(8, 8)
    with pytest.raises(pkg.GLBMError) as e:
        s.step(1)
    assert e.value.name == "GLBM_ESTATE"
    eps, K = media.uniform_medium(8, 8, 0.5, 1e-3)
    bad = eps.copy()
    bad[3, 4] = 1.5
    with pytest.raises(pkg.GLBMError) as e:
        s.set_medium(bad, K)
    assert e.value.name == "GLBM_EINVAL" and "eps" in str(e.value)
    Kn = K.copy()
    Kn[0, 0] = np.nan
    with pytest.raises(pkg.GLBMError):
        s.set_medium(eps, Kn)
    import torch
    with pytest.raises(pkg.GLBMError):  # device-side validation
        s.set_medium(torch.from_numpy(bad).cuda(), torch.from_numpy(K).cuda())
    s.set_medium(eps, K)
    with pytest.raises(pkg.GLBMError) as e:
        s.mean_velocity()
    assert e.value.name == "GLBM_ESTATE"
    with pytest.raises(pkg.GLBMError):
        s.permeability()  # G_x = 0
    done, conv = s.step(0)
    assert done == 0 and not conv


def test_nan_detected(pkg):
    """A non-finite force drives the state to NaN; the device reduction flags
    it and the call returns GLBM_ENAN with the state kept (no GPU fault)."""
    eps, K = media.uniform_medium(16, 8, 1.0, math.inf)
    s = pkg.Solver(16, 8)
    s.set_medium(eps, K)
    s.set_force(1e300, 0.0)
    with pytest.raises(pkg.GLBMError) as e:
        s.step(200, tol=1e-9, check_every=10)
    assert e.value.name == "GLBM_ENAN"


@pytest.mark.parametrize("storage", ["f32", "f64", "f16", "bf16"])
def test_graph_replay_matches_direct_launches(pkg, storage):
    """On a user stream glbm_step replays captured chunk graphs; the result
    equals direct launches on the legacy stream bit for bit, including odd
    chunk lengths, a partial last chunk and convergence tests.  16-bit
    storage takes its stochastic-rounding key from a device step counter
    inside graphs and from the host otherwise: the keys, hence the bits,
    agree (its launch count differs by the counter updates)."""
    import torch
    eps, K, _ = media.two_phase_medium(96, 40, seed=8)
    out = []
    for stream in (None, torch.cuda.Stream()):
        s = pkg.Solver(96, 40, storage=storage, stream=stream)
        s.set_medium(eps, K)
        s.set_force(1e-6)
        s.step(250, check_every=7)
        a = s.step(1000, tol=1e-12, check_every=50)
        s.set_force(2e-6)
        s.step(33, check_every=10)
        if stream is not None:
            stream.synchronize()
        out.append((s.distributions(), s.mean_velocity(), a, s.counters()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
    if storage in ("f32", "f64"):
        assert out[0][3] == out[1][3]
    else:
        assert out[0][3][0] == out[1][3][0]


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_dependent_launch_matches_plain_launches(pkg, storage):
    """On a user stream the step kernels use programmatic dependent launch
    (the next step is placed while the previous drains and waits on the GPU
    for it); on the legacy stream they launch plainly.  This compares the
    two bit for bit on a lattice of several waves of blocks (on the user
    stream the 100-step chunks are replayed graphs)."""
    import torch
    eps, K, _ = media.two_phase_medium(512, 384, seed=12)
    out = []
    for stream in (None, torch.cuda.Stream()):
        s = pkg.Solver(512, 384, storage=storage, stream=stream)
        s.set_medium(eps, K)
        s.set_force(1e-5)
        s.step(400, check_every=100)
        if stream is not None:
            stream.synchronize()
        out.append((s.distributions(), s.mean_velocity()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
