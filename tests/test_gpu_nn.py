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


@pytest.mark.parametrize("h,w", [(8, 12), (7, 9), (20, 70)], ids=["aligned", "ragged", "tiles"])
def test_elementwise_kernels_on_channel_slices(env, h, w):
    """ReLU mask, channel copy, 2x2 pooling and nearest upsampling, forward
    and backward, on a 3-channel slice (channels 1-3) of 5-channel tensors,
    against NumPy in the kernels' FP32 operation order: bit for bit.  hw a
    multiple of 4 with 16-byte aligned planes takes the float4 path, the
    others the scalar one; (20, 70) spans several 32 x 8 pixel tiles."""
    pkg, _, torch = env
    lib = pkg.load()
    rng = np.random.default_rng(h * 100 + w)
    n, c, C5 = 2, 3, 5
    f32 = np.float32

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=f32)).cuda()

    def sl(t, hh, ww):  # pointer to channel 1 of a (n, 5, hh, ww) tensor, sample stride
        return t.data_ptr() + 4 * hh * ww, C5 * hh * ww

    # ReLU backward: dy = 0 where y <= 0 (also NaN)
    y = rng.normal(size=(n, C5, h, w)).astype(f32)
    y[0, 1, 0, 0] = np.nan
    dy = rng.normal(size=(n, C5, h, w)).astype(f32)
    ty, tdy = dev(y), dev(dy)
    assert lib.glbm_nn_relu_bwd(*sl(ty, h, w), *sl(tdy, h, w), c, n, h, w, None) == 0
    want = dy.copy()
    want[:, 1:4] = np.where(y[:, 1:4] > 0, dy[:, 1:4], f32(0))
    torch.cuda.synchronize()
    assert np.array_equal(tdy.cpu().numpy(), want)

    # channel copy, plain and accumulating
    src = rng.normal(size=(n, C5, h, w)).astype(f32)
    dst = rng.normal(size=(n, C5, h, w)).astype(f32)
    ts, td = dev(src), dev(dst)
    assert lib.glbm_nn_copy_channels(*sl(ts, h, w), *sl(td, h, w), c, n, h, w, 1, None) == 0
    want = dst.copy()
    want[:, 1:4] = dst[:, 1:4] + src[:, 1:4]
    torch.cuda.synchronize()
    assert np.array_equal(td.cpu().numpy(), want)
    assert lib.glbm_nn_copy_channels(*sl(ts, h, w), *sl(td, h, w), c, n, h, w, 0, None) == 0
    want[:, 1:4] = src[:, 1:4]
    torch.cuda.synchronize()
    assert np.array_equal(td.cpu().numpy(), want)

    # nearest upsampling h x w -> 2h x 2w and its adjoint
    x = rng.normal(size=(n, C5, h, w)).astype(f32)
    up = rng.normal(size=(n, C5, 2 * h, 2 * w)).astype(f32)
    tx, tu = dev(x), dev(up)
    assert lib.glbm_nn_upsample2(*sl(tx, h, w), *sl(tu, 2 * h, 2 * w), c, n, h, w, 0, None) == 0
    want = up.copy()
    want[:, 1:4] = x[:, 1:4].repeat(2, axis=2).repeat(2, axis=3)
    torch.cuda.synchronize()
    assert np.array_equal(tu.cpu().numpy(), want)
    g = rng.normal(size=(n, C5, 2 * h, 2 * w)).astype(f32)
    dx = rng.normal(size=(n, C5, h, w)).astype(f32)
    tg, tdx = dev(g), dev(dx)
    assert lib.glbm_nn_upsample2(*sl(tg, 2 * h, 2 * w), *sl(tdx, h, w), c, n, h, w, 1, None) == 0
    want = dx.copy()
    gs = g[:, 1:4]
    want[:, 1:4] = (gs[..., 0::2, 0::2] + gs[..., 0::2, 1::2]) + (gs[..., 1::2, 0::2] + gs[..., 1::2, 1::2])
    torch.cuda.synchronize()
    assert np.array_equal(tdx.cpu().numpy(), want)

    # 2x2 average pooling 2h x 2w -> h x w and its adjoint (accumulating)
    big = rng.normal(size=(n, C5, 2 * h, 2 * w)).astype(f32)
    small = rng.normal(size=(n, C5, h, w)).astype(f32)
    tb, tsm = dev(big), dev(small)
    assert lib.glbm_nn_pool2(*sl(tb, 2 * h, 2 * w), *sl(tsm, h, w), c, n, 2 * h, 2 * w, 0, 0, None) == 0
    want = small.copy()
    bs = big[:, 1:4]
    want[:, 1:4] = f32(0.25) * ((bs[..., 0::2, 0::2] + bs[..., 0::2, 1::2]) + (bs[..., 1::2, 0::2] + bs[..., 1::2, 1::2]))
    torch.cuda.synchronize()
    assert np.array_equal(tsm.cpu().numpy(), want)
    pooled = want  # now the pooling backward's input (dy)
    acc = rng.normal(size=(n, C5, 2 * h, 2 * w)).astype(f32)
    ta = dev(acc)
    assert lib.glbm_nn_pool2(*sl(tsm, h, w), *sl(ta, 2 * h, 2 * w), c, n, 2 * h, 2 * w, 1, 1, None) == 0
    want = acc.copy()
    want[:, 1:4] = acc[:, 1:4] + (f32(0.25) * pooled[:, 1:4]).repeat(2, axis=2).repeat(2, axis=3)
    torch.cuda.synchronize()
    assert np.array_equal(ta.cpu().numpy(), want)
