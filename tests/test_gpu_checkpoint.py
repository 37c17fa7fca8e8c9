"""Checkpoint and resume (glbm_save / glbm_load): a run saved at step k and
continued in a fresh handle gives the same bits as the run that never
stopped, for every storage format, with and without the Forchheimer term
and with convergence tests spanning the save."""

import os

import numpy as np
import pytest

import media

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1601_00704_gb300 import build
    build.build()
    import paper_1601_00704_gb300 as p
    return p


@pytest.mark.parametrize("storage,feps,user_stream", [
    ("f32", 0.0, True), ("f32", -1.0, False), ("f64", 0.0, True),
    ("f16", 0.0, True), ("bf16", 0.0, True), ("bf16", 0.0, False)])
def test_resume_is_bitwise(pkg, tmp_path, storage, feps, user_stream):
    import torch
    nx, ny = 96, 40
    eps, K, _ = media.two_phase_medium(nx, ny, seed=21)
    stream = torch.cuda.Stream() if user_stream else None
    path = os.fspath(tmp_path / "run.ckpt")

    def solver():
        return pkg.Solver(nx, ny, storage=storage, stream=stream)

    a = solver()
    a.set_medium(eps, K, feps)
    a.set_force(2e-5, 1e-6)
    a.step(300, tol=1e-12, check_every=100)
    a.save(path)
    r1 = a.step(450, tol=1e-12, check_every=50)
    want = (a.distributions(), a.mean_velocity(), a.counters()[0])

    b = solver()  # no set_medium: the checkpoint carries the medium
    b.load(path)
    r2 = b.step(450, tol=1e-12, check_every=50)
    got = (b.distributions(), b.mean_velocity(), b.counters()[0])
    assert r1 == r2
    assert np.array_equal(want[0], got[0])
    assert np.array_equal(want[1], got[1])
    assert want[2] == got[2]


def test_load_rejects_mismatch_and_corruption(pkg, tmp_path):
    eps, K, _ = media.two_phase_medium(64, 32, seed=2)
    a = pkg.Solver(64, 32)
    a.set_medium(eps, K)
    a.set_force(1e-6)
    a.step(20)
    path = tmp_path / "a.ckpt"
    a.save(os.fspath(path))
    for other in (pkg.Solver(64, 33), pkg.Solver(64, 32, storage="bf16"),
                  pkg.Solver(64, 32, tau=0.8), pkg.Solver(64, 32, walls=False)):
        with pytest.raises(pkg.GLBMError) as e:
            other.load(os.fspath(path))
        assert e.value.name == "GLBM_EINVAL"
    data = bytearray(path.read_bytes())
    data[-5] ^= 0x40
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(data))
    b = pkg.Solver(64, 32)
    with pytest.raises(pkg.GLBMError) as e:
        b.load(os.fspath(bad))
    assert "checksum" in str(e.value)
    (tmp_path / "short.ckpt").write_bytes(bytes(data[:100]))
    with pytest.raises(pkg.GLBMError):
        b.load(os.fspath(tmp_path / "short.ckpt"))
    with pytest.raises(pkg.GLBMError) as e:
        pkg.Solver(64, 32).save(os.fspath(tmp_path / "none.ckpt"))
    assert e.value.name == "GLBM_ESTATE"
