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


def test_phase_threshold_equals_stable_sort_definition():
    """OM = the round(phi*N) largest field values, ties to the lowest index."""
    for seed in range(3):
        rng = np.random.Generator(np.random.PCG64(seed))
        om = media.two_phase_map(96, 80, 0.3, 6, rng)
        rng = np.random.Generator(np.random.PCG64(seed))
        f = media.gaussian_random_field(96, 80, 6, rng).ravel()
        order = np.argsort(-f, kind="stable")
        want = np.zeros(f.size, bool)
        want[order[:round(0.3 * f.size)]] = True
        assert np.array_equal(om.ravel(), want)
    f = np.array([1.0, 2.0, 2.0, 2.0, 0.5])  # exact ties: lowest index first
    thr_mask = np.zeros(5, bool)
    thr = np.partition(f, 5 - 2)[5 - 2]
    thr_mask = f > thr
    ties = np.flatnonzero(f == thr)
    thr_mask[ties[:2 - int(thr_mask.sum())]] = True
    assert thr_mask.tolist() == [False, True, True, False, False]


def test_shale_batch_recipe():
    b = media.shale_batch(6, seed=1)
    assert len(b) == 6
    for m in b:
        assert m["n"] % 64 == 0 and 64 <= m["n"] <= 1024
        assert m["r"].shape == (m["n"], m["n"]) and (m["r"] > 0).all()
        assert 0.5e6 <= m["P"] <= 30e6 and 2e6 <= m["P_L"] <= 10e6
        assert 0.002 <= m["V_L"] <= 0.01
        assert abs(np.median(m["r"][m["organic"]]) / 5e-9 - 1) < 0.2
