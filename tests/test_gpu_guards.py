"""Memory safety of the solver's and the batch's kernels without a sanitizer:
every device buffer of a handle sits between 4 KB guard zones of a fixed
byte pattern (glbm_debug_guards).  After runs that touch every kernel and
copy of the path -- vector, scalar and ragged rows, walls and periodic
boundaries, every storage, Forchheimer coefficients, reductions and
convergence tests, graph replay, host and device inputs, read-back,
checkpoint and resume, the persistent batch kernel -- no guard byte may
have changed.  A poked byte shows that the count sees damage."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1601_00704_gb300 import build
    build.build()
    import paper_1601_00704_gb300 as p
    p.load()
    return p


def _medium(ny, nx, seed):
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.1, 0.9, (ny, nx))
    K = 10.0 ** rng.uniform(-3, 0, (ny, nx))
    return eps, K


# (nx, ny): vector rows, scalar rows (nx not a multiple of 4), a ragged wide
# lattice, and the smallest lattice
SHAPES = [(64, 48), (67, 33), (1030, 17), (2, 2)]


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("walls", [True, False], ids=["walls", "periodic"])
def test_solver_writes_stay_in_bounds(pkg, tmp_path, storage, nx, ny, walls):
    import torch
    eps, K = _medium(ny, nx, nx * 131 + ny)
    stream = torch.cuda.Stream()
    with pkg.Solver(nx, ny, tau=0.9, storage=storage, walls=walls, stream=stream) as s:
        assert s.guard_damage() == 0
        s.set_medium(eps, K, F_eps=0.5)
        s.set_force(1e-5, 2e-6)
        s.step(30, tol=1e-12, check_every=10)
        s.step(7)
        s.mean_velocity()
        s.permeability()
        s.velocity()
        s.distributions()
        path = str(tmp_path / "ck.glbm")
        s.save(path)
        s.step(5)
        s.load(path)
        s.step(12, tol=1e-12, check_every=4)
        rng = np.random.default_rng(1)
        s.init_equilibrium(1.0 + 1e-3 * rng.standard_normal((ny, nx)), 1e-4 * rng.standard_normal((ny, nx)),
                           np.zeros((ny, nx)))
        s.step(9, tol=1e-12, check_every=3)
        dev_eps = torch.from_numpy(eps).cuda()
        dev_K = torch.from_numpy(K).cuda()
        s.set_medium(dev_eps, dev_K)
        s.step(6)
        assert s.guard_damage() == 0
        assert s.guard_damage(poke=True) == 1
        assert s.guard_damage() == 0


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("persistent", [False, True], ids=["graphs", "persistent"])
def test_batch_writes_stay_in_bounds(pkg, storage, persistent):
    shapes = [(20, 16), (33, 64), (7, 4), (64, 128)]
    b = pkg.Batch(shapes, tau=0.9, storage=storage, walls=True)
    try:
        assert b.guard_damage() == 0
        for i, (ny, nx) in enumerate(shapes):
            b.set_medium(i, *_medium(ny, nx, 7 + i))
        b.set_force(1e-5)
        b.set_persistent(persistent)
        b.step(40, tol=1e-12, check_every=10)
        b.results()
        for i in range(len(shapes)):
            b.fields(i)
        assert b.guard_damage() == 0
        assert b.guard_damage(poke=True) == 1
        assert b.guard_damage() == 0
    finally:
        b.close()
