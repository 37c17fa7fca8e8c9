"""Pins of the FP64 U-Net oracle against mathematics independent of it:
finite differences of the loss, a library correlation, adjoint identities
and a closed-form property of Adam."""

import numpy as np
import pytest

from oracle import unet as U

LEVELS, BASE = 3, 2


def tiny(seed=0):
    rng = np.random.default_rng(seed)
    specs = U.layer_specs(2, 2, BASE, LEVELS)
    total = sum(co * ci * k * k + co for _, ci, co, k in specs)
    flat = rng.normal(0, 0.5, total)
    x = rng.normal(0, 1, (2, 2, 8, 8))
    t = rng.normal(0, 1, (2, 2, 8, 8))
    return specs, flat, x, t


def loss_of(flat, specs, x, t, cw=(1.0, 0.5)):
    y, _ = U.forward(U.unpack(flat, specs), x, LEVELS)
    return U.mse(y, t, cw)[0]


def test_gradients_match_finite_differences():
    specs, flat, x, t = tiny()
    params = U.unpack(flat, specs)
    y, cache = U.forward(params, x, LEVELS)
    L, gy = U.mse(y, t, (1.0, 0.5))
    grads, gx = U.backward(params, cache, gy, LEVELS)
    g = U.pack(grads, specs)
    rng = np.random.default_rng(1)
    h = 1e-6
    off = 0
    for name, ci, co, k in specs:
        n = co * ci * k * k + co
        for idx in rng.choice(n, size=min(4, n), replace=False):
            i = off + idx
            p, m = flat.copy(), flat.copy()
            p[i] += h
            m[i] -= h
            fd = (loss_of(p, specs, x, t) - loss_of(m, specs, x, t)) / (2 * h)
            assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), (name, idx)
        off += n
    for idx in [(0, 0, 3, 4), (1, 1, 7, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (loss_of(flat, specs, xp, t) - loss_of(flat, specs, xm, t)) / (2 * h)
        assert gx[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_conv_is_zero_padded_correlation():
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 1, 9, 7))
    W = rng.normal(size=(1, 1, 3, 3))
    y = U.conv(x, W, np.zeros(1))
    ref = scipy_signal.correlate2d(x[0, 0], W[0, 0], mode="same", boundary="fill")
    np.testing.assert_allclose(y[0, 0], ref, rtol=1e-13, atol=1e-13)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 3, 8, 6))
    z = rng.normal(size=(2, 3, 4, 3))
    assert np.sum(U.pool(x) * z) == pytest.approx(np.sum(x * U.pool_backward(z)), rel=1e-13)
    assert np.sum(U.up(z) * x) == pytest.approx(np.sum(z * U.up_backward(x)), rel=1e-13)


def test_adam_constant_gradient_moves_lr_per_step():
    """With a constant gradient the bias-corrected moments equal g and g^2,
    so each step moves each parameter by lr * g / (|g| + eps)."""
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 4.0])
    m = np.zeros(3)
    v = np.zeros(3)
    q = p
    for t in range(1, 6):
        q, m, v = U.adam(q, g, m, v, t, lr=0.01)
    np.testing.assert_allclose(q, p - 5 * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-10)


def test_pool_hand_computed_averages():
    """2x2 average pooling of 0..15 laid out row by row in a 4x4 image: each
    output is the average of its block, written out by hand (a sum pool
    gives 4x these; a max pool gives the blocks' last entries)."""
    x = np.arange(16, dtype=np.float64).reshape(1, 1, 4, 4)
    x = np.concatenate([x, 10 * x], axis=1)  # a second channel, scaled
    expect = np.array([[(0 + 1 + 4 + 5) / 4, (2 + 3 + 6 + 7) / 4],
                       [(8 + 9 + 12 + 13) / 4, (10 + 11 + 14 + 15) / 4]])
    assert expect.tolist() == [[2.5, 4.5], [10.5, 12.5]]
    y = U.pool(x)
    np.testing.assert_array_equal(y[0, 0], expect)
    np.testing.assert_array_equal(y[0, 1], 10 * expect)


def test_pool_backward_hand_computed():
    """The gradient of an average pool spreads each output gradient over its
    2x2 block with weight 1/4 (a pool_backward without the 1/4 fails)."""
    dy = np.array([[1.0, 2.0], [3.0, 4.0]]).reshape(1, 1, 2, 2)
    expect = np.array([[0.25, 0.25, 0.5, 0.5],
                       [0.25, 0.25, 0.5, 0.5],
                       [0.75, 0.75, 1.0, 1.0],
                       [0.75, 0.75, 1.0, 1.0]])
    np.testing.assert_array_equal(U.pool_backward(dy)[0, 0], expect)
    # nearest upsampling copies, and its adjoint sums the four copies
    np.testing.assert_array_equal(U.up(dy)[0, 0], 4 * expect)
    np.testing.assert_array_equal(U.up_backward(U.up(dy)), 4 * dy)


def test_mse_hand_computed():
    """Weighted MSE on 2 samples x 2 channels of 4x4 pixels with a constant
    error per (sample, channel): channel 0 errors 1 and 3, channel 1 errors 2
    and 0, channel weights (1, 0.5).  Per channel the mean over samples and
    pixels of the squared error is (1 + 9)/2 = 5 and (4 + 0)/2 = 2, so the
    loss is 1*5 + 0.5*2 = 6.  A mean over channels too gives 3, a dropped
    channel weight gives 7."""
    d = np.zeros((2, 2, 4, 4))
    d[0, 0], d[1, 0], d[0, 1], d[1, 1] = 1.0, 3.0, 2.0, 0.0
    target = np.random.default_rng(5).normal(size=d.shape)
    loss, grad = U.mse(target + d, target, (1.0, 0.5))
    assert loss == pytest.approx(6.0, rel=1e-14)
    # d loss / d pred = 2 w_c d / (samples * pixels) = w_c d / 16 here
    np.testing.assert_allclose(grad[0, 0], np.full((4, 4), 1.0 / 16), rtol=1e-14)
    np.testing.assert_allclose(grad[1, 0], np.full((4, 4), 3.0 / 16), rtol=1e-14)
    np.testing.assert_allclose(grad[0, 1], np.full((4, 4), 0.5 * 2.0 / 16), rtol=1e-14)
    np.testing.assert_array_equal(grad[1, 1], np.zeros((4, 4)))
