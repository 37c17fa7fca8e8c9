"""The seeded synthetic media: deterministic, exact phase fraction, ranges."""

import numpy as np

import media


def test_two_phase_medium_recipe():
    eps, K, om = media.two_phase_medium(128, 128, om_fraction=0.2,
                                        corr_len=8, seed=0)
    assert eps.shape == K.shape == om.shape == (128, 128)
    assert om.sum() == round(0.2 * 128 * 128)
    assert set(np.unique(eps)) == {0.10, 0.15}
    assert np.all(eps[om] == 0.15) and np.all(eps[~om] == 0.10)
    assert K[om].min() >= 5e-4 and K[om].max() <= 5e-3
    assert K[~om].min() >= 1e-4 and K[~om].max() <= 1e-3
    # log-uniform: log10 K spreads evenly over its decade
    lk = np.log10(K[~om])
    assert abs(lk.mean() - (-3.5)) < 0.02
    eps2, K2, om2 = media.two_phase_medium(128, 128, seed=0)
    assert np.array_equal(K, K2) and np.array_equal(om, om2)
    _, K3, _ = media.two_phase_medium(128, 128, seed=1)
    assert not np.array_equal(K, K3)


def test_clusters_grow_with_correlation_length():
    """OM forms clusters: the fraction of OM nodes whose right neighbour is
    also OM rises with the correlation length (0.2 for white noise)."""
    fr = []
    for ell in (1, 4, 16):
        _, _, om = media.two_phase_medium(256, 256, corr_len=ell, seed=3)
        fr.append((om & np.roll(om, -1, axis=1)).sum() / om.sum())
    assert fr[0] < fr[1] < fr[2] and fr[2] > 0.9


def test_layered_and_uniform():
    eps, K = media.layered_medium(10, 3, [(4, 0.1, 1.0), (6, 0.2, 2.0)], "x")
    assert np.all(K[:, :4] == 1.0) and np.all(K[:, 4:] == 2.0)
    e, k = media.uniform_medium(3, 2, 0.5, np.inf)
    assert np.all(np.isinf(k)) and np.all(e == 0.5)
