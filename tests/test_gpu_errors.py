"""Error paths of the graph-captured chunks, driven by the library's host-side
test hook (glbm_debug_fail_launch), which refuses a chosen kernel launch on
the host without calling CUDA: nothing faults on the GPU.

A refusal while a chunk is being captured must end and discard the capture,
return GLBM_ECUDA and leave the handle exactly as it was before that chunk:
same distributions, step count and launch count, and a later run that
continues from there is bitwise the run that never failed.
"""

import numpy as np
import pytest

import media

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1601_00704_gb300 import build
    build.build()
    import torch

    import paper_1601_00704_gb300 as pkg
    lib = pkg.load()
    yield pkg, lib, torch
    lib.glbm_debug_fail_launch(-1)


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("after", [0, 17, 64])  # first step, a middle step, the finalize
def test_failed_capture_leaves_solver_unchanged(env, storage, after):
    pkg, lib, torch = env
    eps, K, _ = media.two_phase_medium(96, 40, seed=3)
    stream = torch.cuda.Stream()

    def fresh():
        s = pkg.Solver(96, 40, storage=storage, stream=stream)
        s.set_medium(eps, K)
        s.set_force(1e-5)
        s.step(120, check_every=60)  # a captured 60-step chunk, replayed once
        return s

    s = fresh()
    f0, c0 = s.distributions(), s.counters()
    lib.glbm_debug_fail_launch(after)
    try:
        with pytest.raises(pkg.GLBMError) as e:
            s.step(64, check_every=64)  # a new chunk length: captured now, refused inside
    finally:
        lib.glbm_debug_fail_launch(-1)
    assert e.value.name == "GLBM_ECUDA" and "injected" in str(e.value)
    assert s.counters() == c0
    assert np.array_equal(s.distributions(), f0)
    s.step(64, check_every=64)
    ref = fresh()
    ref.step(64, check_every=64)
    stream.synchronize()
    assert np.array_equal(s.distributions(), ref.distributions())
    assert np.array_equal(s.mean_velocity(), ref.mean_velocity())
    # (launch counts differ by the two exports of the failed handle)
    assert s.counters()[0] == ref.counters()[0]


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_failed_capture_leaves_batch_unchanged(env, storage):
    pkg, lib, torch = env
    shapes = [(24, 32), (40, 64), (16, 16)]
    meds = [media.two_phase_medium(nx, ny, seed=i)[:2] for i, (ny, nx) in enumerate(shapes)]

    def fresh():
        b = pkg.Batch(shapes, storage=storage)
        for i, (eps, K) in enumerate(meds):
            b.set_medium(i, eps, K)
        b.set_force(1e-5)
        b.step(50, check_every=50)
        return b

    b = fresh()
    f0 = [b.distributions(i) for i in range(len(shapes))]
    l0 = b.info()["launches"]
    lib.glbm_debug_fail_launch(9)
    try:
        with pytest.raises(pkg.GLBMError) as e:
            b.step(30, check_every=30)
    finally:
        lib.glbm_debug_fail_launch(-1)
    assert e.value.name == "GLBM_ECUDA"
    assert b.info()["launches"] == l0
    for i in range(len(shapes)):
        assert np.array_equal(b.distributions(i), f0[i])
    b.step(30, check_every=30)
    ref = fresh()
    ref.step(30, check_every=30)
    for i in range(len(shapes)):
        assert np.array_equal(b.distributions(i), ref.distributions(i))
    assert np.array_equal(b.results()["kxx"], ref.results()["kxx"])
