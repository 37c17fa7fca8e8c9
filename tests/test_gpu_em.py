"""GPU EM (glbm_em_gmm1d) against the FP64 oracle: both FP64, reductions in
different orders, so parameters agree to ~1e-12 relative after tens of
iterations (bound 1e-9)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1601_00704_gb300 import build
    build.build()
    import paper_1601_00704_gb300 as p
    return p


def test_em_single_sample_collapses(pkg, orc):
    """One sample: the first iteration puts mu on it with zero variance (the
    sample moments); the next E-step is undefined, reported as ENAN."""
    x = np.array([3.25])
    a = pkg.em_gmm1d(x, [1.0], [0.0], [1.0], max_iter=1, tol=0.0)
    b = orc.em_gmm1d(x, [1.0], [0.0], [1.0], max_iter=1, tol=0.0)
    assert a[1][0] == b[1][0] == 3.25 and a[2][0] == b[2][0] == 0.0 and a[0][0] == 1.0
    with pytest.raises(pkg.GLBMError) as e:
        pkg.em_gmm1d(x, [1.0], [0.0], [1.0], max_iter=3, tol=0.0)
    assert e.value.name == "GLBM_ENAN"


@pytest.mark.parametrize("m,k", [(2, 1), (777, 2), (100003, 2), (50000, 3)])
def test_em_matches_oracle(pkg, orc, m, k):
    rng = np.random.default_rng(m + k)
    comps = [(10.0, 1.0, 0.25), (20.0, 4.0, 0.5), (35.0, 2.0, 0.25)][:k]
    w = np.array([c[2] for c in comps])
    w /= w.sum()
    lab = rng.choice(k, size=m, p=w)
    x = np.array([comps[j][0] for j in lab]) + rng.standard_normal(m) * np.array([comps[j][1] for j in lab])
    init = (np.full(k, 1.0 / k), np.linspace(x.min() + 1, x.max() - 1, k), np.full(k, max(x.var(), 1.0)))
    for it in (1, 5, 40):
        a = pkg.em_gmm1d(x, *init, max_iter=it, tol=0.0)
        b = orc.em_gmm1d(x, *init, max_iter=it, tol=0.0)
        assert a[3] == b[3] == it
        for u, v in zip(a[:3], b[:3]):
            np.testing.assert_allclose(u, v, rtol=1e-9, atol=1e-12)
        assert a[4] == pytest.approx(b[4], rel=1e-12)


def test_em_device_input_and_tolerance(pkg, orc):
    import torch
    rng = np.random.default_rng(5)
    z = rng.random(20000) < 0.25
    x = np.where(z, rng.normal(10, 1, 20000), rng.normal(20, 4, 20000))
    a = pkg.em_gmm1d(torch.from_numpy(x).cuda(), [0.5, 0.5], [5.0, 25.0], [9.0, 9.0], max_iter=1000, tol=1e-12)
    b = orc.em_gmm1d(x, [0.5, 0.5], [5.0, 25.0], [9.0, 9.0], max_iter=1000, tol=1e-12)
    assert abs(a[3] - b[3]) <= 1
    np.testing.assert_allclose(a[1], b[1], rtol=1e-8)
    with pytest.raises(pkg.GLBMError):
        pkg.em_gmm1d(x, [0.5, 0.0], [5.0, 25.0], [9.0, 9.0])
