"""FP64 NumPy oracle of the warm-start U-Net (forward, backward, Adam).

TEST INFRASTRUCTURE, NOT PRODUCT CODE: used only by tests/ to check the CUDA
network kernels.  The paper has no surrogate network; this follows the
standard definitions:

* convolution with zero padding k//2:
  y[n,o,h,w] = b[o] + sum_{c,i,j} W[o,c,i,j] x[n,c,h+i-k//2,w+j-k//2];
  its gradients are dW[o,c,i,j] = sum_{n,h,w} dy[n,o,h,w] x_pad[n,c,h+i,w+j],
  db[o] = sum dy[n,o], dx = the adjoint (scatter of W^T dy);
* 2x2 average pooling and 2x nearest upsampling (adjoint of each other up
  to the factor 4);
* ReLU; per-channel weighted mean-squared error; Adam with bias correction.

Architecture (identical parameter order to the CUDA module): encoder levels
l = 0..L-1 with channels base*2^l, each two 3x3 convolutions + ReLU and a
2x2 average pool between levels; decoder levels l = L-2..0, each taking
concat(upsample(previous), encoder l) through two 3x3 convolutions + ReLU;
a 1x1 head without activation.

Pins (tests/test_oracle_unet.py): finite differences of the loss for every
parameter tensor and for the input; single-channel convolution against
scipy.signal.correlate2d; pooling/upsampling adjointness; hand-computed
values of the pool, its gradient and the weighted loss on 4x4 arrays (these
fail for a sum pool, a gradient without its 1/4, a loss averaged over the
channels too or one without its channel weights).
"""

from __future__ import annotations

import numpy as np


def layer_specs(in_ch, out_ch, base, levels):
    """[(name, cin, cout, k)] in parameter order."""
    ch = [base * 2 ** l for l in range(levels)]
    specs = []
    cin = in_ch
    for l in range(levels):
        specs += [(f"e{l}a", cin, ch[l], 3), (f"e{l}b", ch[l], ch[l], 3)]
        cin = ch[l]
    for l in range(levels - 2, -1, -1):
        specs += [(f"d{l}a", ch[l + 1] + ch[l], ch[l], 3), (f"d{l}b", ch[l], ch[l], 3)]
    specs.append(("head", ch[0], out_ch, 1))
    return specs


def unpack(flat, specs):
    """Flat parameter vector -> {name: (W, b)} (views), in the CUDA layout:
    per layer W (cout, cin, k, k) then b (cout)."""
    out, off = {}, 0
    for name, cin, cout, k in specs:
        nw = cout * cin * k * k
        W = flat[off:off + nw].reshape(cout, cin, k, k)
        off += nw
        b = flat[off:off + cout]
        off += cout
        out[name] = (W, b)
    return out


def conv(x, W, b):
    k = W.shape[2]
    p = k // 2
    n, c, h, w = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (p, p), (p, p)))
    y = np.zeros((n, W.shape[0], h, w))
    for i in range(k):
        for j in range(k):
            y += np.einsum("oc,nchw->nohw", W[:, :, i, j], xp[:, :, i:i + h, j:j + w])
    return y + b[None, :, None, None]


def conv_backward(x, W, dy):
    k = W.shape[2]
    p = k // 2
    n, c, h, w = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (p, p), (p, p)))
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for i in range(k):
        for j in range(k):
            dW[:, :, i, j] = np.einsum("nohw,nchw->oc", dy, xp[:, :, i:i + h, j:j + w])
            dxp[:, :, i:i + h, j:j + w] += np.einsum("oc,nohw->nchw", W[:, :, i, j], dy)
    return dxp[:, :, p:p + h, p:p + w], dW, dy.sum(axis=(0, 2, 3))


def pool(x):
    n, c, h, w = x.shape
    return x.reshape(n, c, h // 2, 2, w // 2, 2).mean(axis=(3, 5))


def pool_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=2), 2, axis=3) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up_backward(dy):
    n, c, h, w = dy.shape
    return dy.reshape(n, c, h // 2, 2, w // 2, 2).sum(axis=(3, 5))


def relu(x):
    return np.maximum(x, 0.0)


def mse(pred, target, cw):
    """sum_c cw[c] * mean_{n,h,w} (pred - target)^2 and its gradient."""
    n, c, h, w = pred.shape
    d = pred - target
    wgt = np.asarray(cw, dtype=np.float64)[None, :, None, None] / (n * h * w)
    return float(np.sum(wgt * d * d)), 2.0 * wgt * d


def forward(params, x, levels):
    """-> (y, cache) with every activation kept for the backward pass."""
    cache = {"x": x}
    inp = x
    for l in range(levels):
        a = relu(conv(inp, *params[f"e{l}a"]))
        e = relu(conv(a, *params[f"e{l}b"]))
        cache[f"in{l}"], cache[f"a{l}"], cache[f"e{l}"] = inp, a, e
        if l < levels - 1:
            inp = pool(e)
    top = cache[f"e{levels - 1}"]
    for l in range(levels - 2, -1, -1):
        cat = np.concatenate([up(top), cache[f"e{l}"]], axis=1)
        da = relu(conv(cat, *params[f"d{l}a"]))
        d = relu(conv(da, *params[f"d{l}b"]))
        cache[f"cat{l}"], cache[f"da{l}"], cache[f"d{l}"] = cat, da, d
        top = d
    y = conv(top, *params["head"])
    return y, cache


def backward(params, cache, dy, levels):
    """-> ({name: (dW, db)}, dx)."""
    grads = {}
    top = cache["d0"] if levels > 1 else cache["e0"]
    dtop, grads["head"] = None, None
    dtop, dW, db = conv_backward(top, params["head"][0], dy)
    grads["head"] = (dW, db)
    g_e = {}
    g_top = {0: dtop}  # gradient of the decoder output at level l
    for l in range(0, levels - 1):
        gd = g_top[l] * (cache[f"d{l}"] > 0)
        gda, dW, db = conv_backward(cache[f"da{l}"], params[f"d{l}b"][0], gd)
        grads[f"d{l}b"] = (dW, db)
        gda = gda * (cache[f"da{l}"] > 0)
        gcat, dW, db = conv_backward(cache[f"cat{l}"], params[f"d{l}a"][0], gda)
        grads[f"d{l}a"] = (dW, db)
        c_up = gcat.shape[1] - cache[f"e{l}"].shape[1]
        g_e[l] = gcat[:, c_up:].copy()
        gup = up_backward(gcat[:, :c_up])
        if l + 1 == levels - 1:
            g_e[levels - 1] = gup
        else:
            g_top[l + 1] = gup
    if levels == 1:
        g_e[0] = dtop
    g_in = None
    for l in range(levels - 1, -1, -1):
        ge = g_e[l]
        if l < levels - 1:
            ge = ge + pool_backward(g_in)
        ge = ge * (cache[f"e{l}"] > 0)
        ga, dW, db = conv_backward(cache[f"a{l}"], params[f"e{l}b"][0], ge)
        grads[f"e{l}b"] = (dW, db)
        ga = ga * (cache[f"a{l}"] > 0)
        g_in, dW, db = conv_backward(cache[f"in{l}"], params[f"e{l}a"][0], ga)
        grads[f"e{l}a"] = (dW, db)
    return grads, g_in


def pack(grads, specs):
    return np.concatenate([np.concatenate([grads[name][0].ravel(), grads[name][1].ravel()])
                           for name, _, _, _ in specs])


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
