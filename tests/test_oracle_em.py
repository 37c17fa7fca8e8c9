"""Pins of the EM oracle (Sec. 2.2, Eqs. 20-24)."""

import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def table():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "em_two_cluster.txt"))
            if l.strip() and not l.startswith("#")]
    return np.array([[float(v) for v in r[1:]] for r in rows])


def sample(m, seed):
    t = table()
    rng = np.random.default_rng(seed)
    z = rng.random(m) < t[0, 2]
    return np.where(z, rng.normal(t[0, 0], t[0, 1], m), rng.normal(t[1, 0], t[1, 1], m))


def test_recovers_the_papers_test_mixture(orc):
    """From a seeded sample of the table's true mixture, EM recovers the true
    means, deviations and fractions within 5 sampling standard errors."""
    t = table()
    m = 20000
    phi, mu, var, it, _ = orc.em_gmm1d(sample(m, 0), [0.5, 0.5], [5.0, 25.0], [9.0, 9.0],
                                       max_iter=1000, tol=1e-13)
    sd = np.sqrt(var)
    for j in range(2):
        mj = m * t[j, 2]
        assert abs(mu[j] - t[j, 0]) < 5 * t[j, 1] / np.sqrt(mj)
        assert abs(sd[j] - t[j, 1]) < 5 * t[j, 1] / np.sqrt(2 * mj)
        assert abs(phi[j] - t[j, 2]) < 5 * np.sqrt(t[j, 2] * (1 - t[j, 2]) / m)
    # the paper's own estimates lie within 3 standard errors of the truth for
    # a sample of the order of a thousand points
    for j in range(2):
        se = t[j, 1] / np.sqrt(1000 * t[j, 2])
        assert abs(t[j, 3] - t[j, 0]) < 3 * se


def test_single_component_is_the_sample_moments(orc):
    """k = 1: every responsibility is 1, so one M-step gives the sample mean
    and the biased sample variance."""
    x = np.random.default_rng(2).normal(3.0, 2.0, 5000)
    phi, mu, var, it, _ = orc.em_gmm1d(x, [1.0], [0.0], [1.0], max_iter=1)
    assert phi[0] == pytest.approx(1.0, abs=1e-15)
    assert mu[0] == pytest.approx(x.mean(), rel=1e-13)
    assert var[0] == pytest.approx(x.var(), rel=1e-12)


def test_loglikelihood_never_decreases(orc):
    """EM's defining property: the likelihood is non-decreasing."""
    x = sample(4000, 3)
    lls = [orc.em_gmm1d(x, [0.3, 0.7], [8.0, 22.0], [4.0, 4.0], max_iter=t)[4] for t in range(1, 25)]
    assert all(b >= a - 1e-13 for a, b in zip(lls, lls[1:]))
    phi = orc.em_gmm1d(x, [0.3, 0.7], [8.0, 22.0], [4.0, 4.0], max_iter=24)[0]
    assert phi.sum() == pytest.approx(1.0, abs=1e-14)
