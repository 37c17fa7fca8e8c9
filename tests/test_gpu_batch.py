"""Batched media (one launch per step for many lattices) and the DGM/GMS
per-node permeability builder, against single-lattice runs and the oracle."""

import math

import numpy as np
import pytest

import media

pytestmark = pytest.mark.gpu

SHAPES = [(48, 64), (32, 128), (80, 36), (17, 516), (64, 64)]


@pytest.fixture(scope="module")
def pkg():
    from paper_1601_00704_gb300 import build
    build.build()
    import paper_1601_00704_gb300 as p
    return p


def media_for(shapes, seed=0):
    out = []
    for i, (ny, nx) in enumerate(shapes):
        eps, K = media.random_medium(nx, ny, seed=seed + i, k_range=(1e-3, 1e0))
        out.append((eps, K))
    return out


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("walls", [True, False])
def test_batch_matches_single_bitwise(pkg, storage, walls):
    """Each medium of a batch evolves exactly as it would alone (same kernel
    body, same stochastic-rounding keys), across chunks replayed from a
    captured graph."""
    md = media_for(SHAPES)
    b = pkg.Batch(SHAPES, tau=0.8, storage=storage, walls=walls)
    for i, (eps, K) in enumerate(md):
        b.set_medium(i, eps, K)
    b.set_force(2e-5, -5e-6)
    done, left = b.step(37, check_every=10)
    assert done == 37 and left == len(SHAPES)
    res = b.results()
    for i, ((ny, nx), (eps, K)) in enumerate(zip(SHAPES, md)):
        s = pkg.Solver(nx, ny, tau=0.8, storage=storage, walls=walls)
        s.set_medium(eps, K)
        s.set_force(2e-5, -5e-6)
        s.step(37)
        assert np.array_equal(b.distributions(i), s.distributions()), i
        assert res["kxx"][i] == pytest.approx(s.permeability(), rel=1e-13)
        assert res["steps"][i] == 37


def test_schedule_does_not_change_results(pkg):
    md = media_for(SHAPES, seed=5)
    outs = []
    for threads, order in ((64, 0), (256, 2), (128, 1)):
        b = pkg.Batch(SHAPES, storage="bf16")
        for i, (eps, K) in enumerate(md):
            b.set_medium(i, eps, K)
        b.set_force(1e-5)
        b.set_schedule(threads, order)
        b.step(25, check_every=7)
        outs.append([b.distributions(i) for i in range(len(SHAPES))])
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert np.array_equal(a, c)


def test_autotune_picks_a_schedule_and_resets(pkg):
    md = media_for(SHAPES, seed=9)
    b = pkg.Batch(SHAPES)
    for i, (eps, K) in enumerate(md):
        b.set_medium(i, eps, K)
    b.set_force(1e-5)
    t, o = b.autotune(trial_steps=5)
    assert t in (64, 128, 256) and o in (0, 1, 2)
    assert b.info()["threads"] == t
    b.step(12, check_every=12)
    fresh = pkg.Batch(SHAPES)
    for i, (eps, K) in enumerate(md):
        fresh.set_medium(i, eps, K)
    fresh.set_force(1e-5)
    fresh.step(12, check_every=12)
    for i in range(len(SHAPES)):
        assert np.array_equal(b.distributions(i), fresh.distributions(i))


def test_converged_media_leave_the_batch(pkg):
    """Small media converge first, leave the tile table, and keep their state
    while the others run on; results match each medium run alone to its own
    convergence."""
    # clear channels (eps = 1, K = inf): viscous relaxation time ~ H^2 / nu
    shapes = [(8, 8), (16, 16), (48, 64)]
    md = [media.uniform_medium(nx, ny, 1.0, math.inf) for ny, nx in shapes]
    b = pkg.Batch(shapes)
    for i, (eps, K) in enumerate(md):
        b.set_medium(i, eps, K)
    b.set_force(1e-5)
    done, left = b.step(200000, tol=1e-9, check_every=100)
    res = b.results()
    assert left == 0 and res["converged"].all()
    assert len(set(res["steps"].tolist())) > 1
    for i, ((ny, nx), (eps, K)) in enumerate(zip(shapes, md)):
        s = pkg.Solver(nx, ny)
        s.set_medium(eps, K)
        s.set_force(1e-5)
        n, conv = s.step(200000, tol=1e-9, check_every=100)
        assert conv and n == res["steps"][i]
        assert np.array_equal(b.distributions(i), s.distributions())


def test_batch_errors(pkg):
    with pytest.raises(pkg.GLBMError):
        pkg.Batch([(8, 6)])  # nx not a multiple of 4
    with pytest.raises(pkg.GLBMError):
        pkg.Batch([(8, 8)], storage="f16")
    b = pkg.Batch([(8, 8), (8, 12)])
    with pytest.raises(pkg.GLBMError) as e:
        b.step(1)
    assert e.value.name == "GLBM_ESTATE"


def test_kapp_field_matches_oracle(pkg, orc):
    """glbm_kapp_field (simplified algebra on the GPU) equals the oracle's
    literal Eq. 18/19 evaluation node by node."""
    rng = np.random.default_rng(3)
    n = 5000
    r = rng.lognormal(math.log(8e-9), 0.6, n)
    org = rng.random(n) < 0.3
    eps = np.where(org, 0.04, 0.02)
    for P in (0.5e6, 5e6, 30e6):
        args = (P, 350.0, 18.231e-6, 2.0, 3000.0, 1 / 4e6, 1e-8, 7.8125e-9)
        got = pkg.kapp_field(r, org, eps, *args)
        want = orc.kapp_field(r, org, eps, *args)
        np.testing.assert_allclose(got, want, rtol=1e-13)
    assert pkg.qsat_from_langmuir_volume(0.005, 1.65e3, 0.04, 0.2, 0.717) == pytest.approx(
        orc.qsat_from_langmuir_volume(0.005, 1.65e3, 0.04, 0.2, 0.717), rel=1e-15)
    with pytest.raises(pkg.GLBMError):
        pkg.kapp_field(np.zeros(4), np.zeros(4, bool), np.full(4, 0.02), *args)


W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
BF16_ULP = 2.0 ** -7


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("walls", [True, False])
def test_batch_matches_oracle_elementwise(pkg, orc, storage, walls):
    """Every medium of an uneven batch against the FP64 oracle, element by
    element, after 1, 4 and 10 steps: FP32 within the step tolerance of the
    single-lattice parity suite (|df| <= 1e-6 * n * max|g|), BF16 within one
    stochastic rounding (2^-7 relative) per step and population."""
    shapes = [(48, 64), (32, 128), (80, 36), (17, 516)]
    md = media_for(shapes, seed=31)
    b = pkg.Batch(shapes, tau=0.8, storage=storage, walls=walls)
    for i, (eps, K) in enumerate(md):
        b.set_medium(i, eps, K)
    b.set_force(3e-4, -1e-4)
    orcs = []
    for (ny, nx), (eps, K) in zip(shapes, md):
        o = orc.Oracle(nx, ny, tau=0.8, periodic_y=not walls)
        o.set_medium(eps, K)
        o.set_force(3e-4, -1e-4)
        orcs.append(o)
    done = 0
    for n in (1, 3, 6):
        b.step(n, check_every=n)
        done += n
        res = b.results()
        for i, o in enumerate(orcs):
            o.step(n)
            gmax = np.abs(o.f - W[:, None, None]).max()
            tol = (1e-6 if storage == "f32" else 2 * BF16_ULP) * done * gmax
            np.testing.assert_allclose(b.distributions(i), o.f, rtol=0, atol=tol, err_msg=f"medium {i}")
            uref = o.mean_u[0]
            assert abs(res["mean_u"][i][0] - uref) <= (2e-5 if storage == "f32" else 3e-2) * done * abs(uref) + 1e-15


def test_batch_converges_per_medium_like_the_oracle(pkg, orc):
    """Clear channels (eps = 1, K = inf, walls in y) of three widths plus a
    uniform Darcy medium, run with a convergence test until each medium
    leaves the batch on its own: each converged K_app equals the converged
    FP64 oracle's within the FP32 bound 1e-4, narrow channels leave first,
    and the Darcy medium gives K G / nu exactly (K_app = K)."""
    shapes = [(8, 32), (16, 32), (24, 32), (12, 16)]
    b = pkg.Batch(shapes, storage="f32")
    inputs = []
    for i, (ny, nx) in enumerate(shapes):
        if i < 3:
            eps, K = np.ones((ny, nx)), np.full((ny, nx), np.inf)
        else:
            eps, K = media.uniform_medium(nx, ny, 0.4, 2e-2)
        b.set_medium(i, eps, K)
        inputs.append((eps, K))
    b.set_force(1e-6)
    done, left = b.step(200000, tol=1e-10, check_every=100)
    assert left == 0
    res = b.results()
    assert res["converged"].all()
    steps = res["steps"]
    assert steps[0] < steps[1] < steps[2]
    for i, ((ny, nx), (eps, K)) in enumerate(zip(shapes, inputs)):
        o = orc.Oracle(nx, ny)
        o.set_medium(eps, K)
        o.set_force(1e-6)
        o.step(200000, tol=1e-10, check_every=100)
        assert res["kxx"][i] == pytest.approx(o.permeability(), rel=1e-4), i
    # uniform porous medium with walls: Brinkman layers at the walls, Darcy
    # value 2e-2 in the core; the mean lies just below it
    assert 0.8 * 2e-2 < res["kxx"][3] < 2e-2


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("walls", [True, False])
@pytest.mark.parametrize("threads", [64, 256])
def test_persistent_matches_graph_launches(pkg, storage, walls, threads):
    """The persistent variant (one cooperative launch per chunk, grid
    barriers between steps) gives the same bits as one launch per step, over
    odd chunk lengths and a convergence test that removes media mid-run."""
    shapes = SHAPES + [(8, 16), (12, 8)]
    md = media_for(shapes, seed=44)
    outs = []
    for pers in (False, True):
        b = pkg.Batch(shapes, tau=0.8, storage=storage, walls=walls)
        for i, (eps, K) in enumerate(md):
            b.set_medium(i, eps, K)
        b.set_schedule(threads, 0)
        b.set_persistent(pers)
        assert b.persistent == pers
        b.set_force(2e-5, -5e-6)
        b.step(37, check_every=10)
        b.step(400, tol=1e-4, check_every=25)
        res = b.results()
        outs.append(([b.distributions(i) for i in range(len(shapes))], res))
    for a, c in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(a, c)
    for k in ("kxx", "steps", "converged"):
        assert np.array_equal(outs[0][1][k], outs[1][1][k])
