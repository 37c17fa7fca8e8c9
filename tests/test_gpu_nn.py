"""CUDA network kernels (glbm_nn_*) and the U-Net module against the FP64
oracle.  FP32 tolerance: relative 2e-5 of the largest magnitude for single
ops, 5e-4 for the composed network (sums over 10^3-10^5 terms)."""

import numpy as np
import pytest

from oracle import unet as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1601_00704_gb300 import build
    build.build()
    import torch

    import paper_1601_00704_gb300 as pkg
    from paper_1601_00704_gb300 import surrogate
    return pkg, surrogate, torch


def close(a, b, rel):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    np.testing.assert_allclose(a, b, rtol=0, atol=rel * max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("k,cin,cout,h,w", [(3, 3, 5, 17, 23), (3, 20, 33, 32, 16), (1, 32, 3, 16, 48)])
def test_conv_ops_match_oracle(env, k, cin, cout, h, w):
    pkg, _, torch = env
    lib = pkg.load()
    rng = np.random.default_rng(k * 100 + cin)
    n = 2
    x = rng.normal(size=(n, cin, h, w)).astype(np.float32)
    W = (rng.normal(size=(cout, cin, k, k)) / np.sqrt(cin * k * k)).astype(np.float32)
    b = rng.normal(size=cout).astype(np.float32)
    dy = rng.normal(size=(n, cout, h, w)).astype(np.float32)
    tx, tW, tb, tdy = (torch.from_numpy(a).cuda() for a in (x, W, b, dy))
    y = torch.empty((n, cout, h, w), device="cuda")
    dx = torch.empty((n, cin, h, w), device="cuda")
    dW = torch.zeros_like(tW)
    db = torch.zeros_like(tb)
    scratch = torch.empty(W.size, device="cuda")
    P = lambda t: t.data_ptr()
    for relu in (0, 1):
        assert lib.glbm_nn_conv_fwd(P(tx), cin * h * w, cin, P(y), cout * h * w, cout, n, h, w, k,
                                    P(tW), P(tb), relu, None) == 0
        want = U.conv(x.astype(np.float64), W.astype(np.float64), b.astype(np.float64))
        if relu:
            want = np.maximum(want, 0)
        torch.cuda.synchronize()
        close(y.cpu().numpy(), want, 2e-5)
    assert lib.glbm_nn_conv_bwd_data(P(tdy), cout * h * w, cout, P(dx), cin * h * w, cin, n, h, w, k,
                                     P(tW), P(scratch), None) == 0
    assert lib.glbm_nn_conv_bwd_weight(P(tx), cin * h * w, cin, P(tdy), cout * h * w, cout, n, h, w, k,
                                       P(dW), P(db), None) == 0
    gx, gW, gb = U.conv_backward(x.astype(np.float64), W.astype(np.float64), dy.astype(np.float64))
    torch.cuda.synchronize()
    close(dx.cpu().numpy(), gx, 2e-5)
    close(dW.cpu().numpy(), gW, 2e-5)
    close(db.cpu().numpy(), gb, 2e-5)


def test_unet_forward_backward_match_oracle(env):
    pkg, surrogate, torch = env
    net = surrogate.UNet(in_ch=3, out_ch=3, base=4, levels=3, seed=1)
    rng = np.random.default_rng(7)
    x = rng.normal(size=(2, 3, 32, 16)).astype(np.float32)
    t = rng.normal(size=(2, 3, 32, 16)).astype(np.float32)
    cw = (1.0, 0.5, 0.25)
    tx = torch.from_numpy(x).cuda()
    tt = torch.from_numpy(t).cuda()
    y = net.forward(tx)
    loss, gy = net.loss(y, tt, cw)
    net.backward(gy)
    torch.cuda.synchronize()
    flat = net.params.cpu().numpy().astype(np.float64)
    specs = U.layer_specs(3, 3, 4, 3)
    params = U.unpack(flat, specs)
    want_y, cache = U.forward(params, x.astype(np.float64), 3)
    want_loss, want_gy = U.mse(want_y, t.astype(np.float64), cw)
    grads, _ = U.backward(params, cache, want_gy, 3)
    close(y.cpu().numpy(), want_y, 5e-5)
    assert float(loss.item()) == pytest.approx(want_loss, rel=1e-4)
    close(net.grads.cpu().numpy(), U.pack(grads, specs), 5e-4)
    # one Adam step
    p0 = flat.copy()
    net.adam_step(1e-3)
    torch.cuda.synchronize()
    want_p, _, _ = U.adam(p0, U.pack(grads, specs), np.zeros_like(p0), np.zeros_like(p0), 1, 1e-3)
    close(net.params.cpu().numpy(), want_p, 1e-6)


def test_pool_upsample_copy_ops(env):
    pkg, _, torch = env
    lib = pkg.load()
    rng = np.random.default_rng(4)
    x = rng.normal(size=(2, 3, 8, 12)).astype(np.float32)
    tx = torch.from_numpy(x).cuda()
    p = torch.empty((2, 3, 4, 6), device="cuda")
    assert lib.glbm_nn_pool2(tx.data_ptr(), 3 * 96, p.data_ptr(), 3 * 24, 3, 2, 8, 12, 0, 0, None) == 0
    u = torch.empty((2, 3, 16, 24), device="cuda")
    assert lib.glbm_nn_upsample2(tx.data_ptr(), 3 * 96, u.data_ptr(), 3 * 384, 3, 2, 8, 12, 0, None) == 0
    torch.cuda.synchronize()
    close(p.cpu().numpy(), U.pool(x.astype(np.float64)), 1e-6)
    close(u.cpu().numpy(), U.up(x.astype(np.float64)), 0)
    # copy into a channel slice of a 5-channel tensor
    big = torch.zeros((2, 5, 8, 12), device="cuda")
    assert lib.glbm_nn_copy_channels(tx.data_ptr(), 3 * 96, big.data_ptr() + 4 * 2 * 96, 5 * 96,
                                     3, 2, 8, 12, 0, None) == 0
    torch.cuda.synchronize()
    assert np.array_equal(big.cpu().numpy()[:, 2:], x)
    assert not big.cpu().numpy()[:, :2].any()
