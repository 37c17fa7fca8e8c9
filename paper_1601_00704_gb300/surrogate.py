"""Learned warm start for the GLBM time loop.

The slow part of a GLBM run is the relaxation of the pressure (density)
field, which diffuses with D ~ c_s^2 K / nu; the velocity follows it within a
few steps through the local Darcy balance.  A start from the exact steady
velocity with a flat density therefore saves nothing, while a start from the
steady density saves almost all of the run.  The surrogate is a U-Net that
maps the medium (eps, log10 K, G) to the steady density deviation and
velocity; ``glbm_init_equilibrium`` then starts the solver from
f = f_eq(rho_pred, u_pred), and the solver still runs to the same
convergence test, which judges the prediction.  The paper has no surrogate:
this is the library's own addition.

Every computation of the network runs in the library's CUDA kernels
(``glbm_nn_*``): 3x3 / 1x1 convolutions (forward, backward-data,
backward-weight), 2x2 average pooling, nearest upsampling, ReLU, weighted
MSE and Adam, in FP32 for training.  Inference can also run on the tensor
cores (``forward_tc``: tcgen05 implicit-GEMM convolutions on BF16 NHWC
activations, FP32 accumulation).  PyTorch only provides device memory and
the stream.

Normalisation (all inputs/targets dimensionless, O(1)):
  inputs   (eps - 0.05) / 0.05,  (log10 K + 2) / 2,  log10(|G|) + 6
  targets  delta_rho / (G * RHO_SCALE),  u * nu / (K G)  (x and y)
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import GLBMError, load

RHO_SCALE = 0.3


def _ptr(t, offset_floats=0):
    return C.c_void_p(t.data_ptr() + 4 * int(offset_floats))


class UNet:
    """U-Net with ``levels`` resolutions (channels base * 2^l), two 3x3
    convolutions + ReLU per level, average-pool down, nearest-up + skip
    concatenation, and a 1x1 head.  FP32 parameters in one flat device
    vector (layout of ``layer_specs``)."""

    def __init__(self, in_ch=3, out_ch=3, base=32, levels=4, seed=0, max_ch=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.in_ch, self.out_ch, self.base, self.levels = in_ch, out_ch, base, levels
        self.ch = [base * 2 ** l if not max_ch else min(base * 2 ** l, max_ch) for l in range(levels)]
        self.specs = []
        cin = in_ch
        for l in range(levels):
            self.specs += [(f"e{l}a", cin, self.ch[l], 3), (f"e{l}b", self.ch[l], self.ch[l], 3)]
            cin = self.ch[l]
        for l in range(levels - 2, -1, -1):
            self.specs += [(f"d{l}a", self.ch[l + 1] + self.ch[l], self.ch[l], 3),
                           (f"d{l}b", self.ch[l], self.ch[l], 3)]
        self.specs.append(("head", self.ch[0], out_ch, 1))
        self.offsets = {}
        off = 0
        for name, ci, co, k in self.specs:
            self.offsets[name] = (off, off + co * ci * k * k)
            off += co * ci * k * k + co
        self.nparams = off
        rng = np.random.default_rng(seed)
        init = np.zeros(off, dtype=np.float32)
        for name, ci, co, k in self.specs:
            ow, ob = self.offsets[name]
            init[ow:ob] = rng.normal(0.0, np.sqrt(2.0 / (ci * k * k)), co * ci * k * k)
        dev = "cuda"
        self.params = torch.from_numpy(init).to(dev)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self.wscratch = torch.empty(max(co * ci * k * k for _, ci, co, k in self.specs),
                                    dtype=torch.float32, device=dev)
        self._bufs = {}
        self._version = 0     # bumped whenever the parameters change
        self._tc = None       # (version, packed BF16 weights, padded biases)
        self._tc_bufs = {}
        self._train_tc = False  # forward/backward on the tensor cores (set per call)
        self._tct = None      # (version, flipped BF16 weights) for input gradients
        self._xh = {}         # BF16 NHWC copy of each convolution's input (training)
        self._gh = {}         # BF16 NHWC output gradients (training scratch)

    # -- plumbing -----------------------------------------------------------
    def _stream(self):
        return C.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def _ok(self, rc, what):
        if rc != 0:
            raise GLBMError(rc, f"{what} failed: {self.lib.glbm_last_error(None).decode()}")

    def _wb(self, name):
        ow, ob = self.offsets[name]
        return ow, ob

    def _conv(self, x, xbs, cin, y, ybs, cout, n, h, w, k, name, relu, xoff=0, yoff=0):
        if self._train_tc:
            return self._conv_tc(x, cin, y, cout, n, h, w, k, name, relu)
        ow, ob = self._wb(name)
        self._ok(self.lib.glbm_nn_conv_fwd(_ptr(x, xoff), xbs, cin, _ptr(y, yoff), ybs, cout, n, h, w, k,
                                           _ptr(self.params, ow), _ptr(self.params, ob), int(relu),
                                           self._stream()), "conv_fwd")

    def _conv_bwd(self, x, xbs, cin, dy, dybs, cout, n, h, w, k, name, dx=None, dxbs=0):
        if self._train_tc:
            return self._conv_bwd_tc(cin, dy, cout, n, h, w, k, name, dx)
        ow, ob = self._wb(name)
        self._ok(self.lib.glbm_nn_conv_bwd_weight(_ptr(x), xbs, cin, _ptr(dy), dybs, cout, n, h, w, k,
                                                  _ptr(self.grads, ow), _ptr(self.grads, ob),
                                                  self._stream()), "conv_bwd_weight")
        if dx is not None:
            self._ok(self.lib.glbm_nn_conv_bwd_data(_ptr(dy), dybs, cout, _ptr(dx), dxbs, cin, n, h, w, k,
                                                    _ptr(self.params, ow), _ptr(self.wscratch),
                                                    self._stream()), "conv_bwd_data")

    def _relu_bwd(self, y, dy, c, n, h, w):
        self._ok(self.lib.glbm_nn_relu_bwd(_ptr(y), c * h * w, _ptr(dy), c * h * w, c, n, h, w,
                                           self._stream()), "relu_bwd")

    def _buffers(self, n, h, w):
        key = (n, h, w)
        if key in self._bufs:
            return self._bufs[key]
        if h % 2 ** (self.levels - 1) or w % 2 ** (self.levels - 1):
            raise ValueError(f"h, w must be multiples of {2 ** (self.levels - 1)}")
        torch = self.torch
        B = {}

        def z(c, l):
            return torch.empty((n, c, h >> l, w >> l), dtype=torch.float32, device="cuda")
        L = self.levels
        for l in range(L):
            c = self.ch[l]
            for nm in ("a", "e", "ga", "ge"):
                B[f"{nm}{l}"] = z(c, l)
            if l < L - 1:
                B[f"p{l}"] = z(c, l + 1)
                B[f"gp{l}"] = z(c, l + 1)
                cc = self.ch[l + 1] + c
                B[f"cat{l}"] = z(cc, l)
                B[f"gcat{l}"] = z(cc, l)
                for nm in ("da", "d", "gda", "gd"):
                    B[f"{nm}{l}"] = z(c, l)
        B["y"] = z(self.out_ch, 0)
        self._bufs = {key: B}  # keep one shape at a time
        return B

    # -- network ------------------------------------------------------------
    def forward(self, x, tc=False):
        """x: contiguous (n, in_ch, h, w) float32 CUDA tensor -> (n, out_ch, h, w).
        tc: run the convolutions on the tensor cores (BF16 operands, FP32
        accumulation and FP32 NCHW activations between layers), keeping what
        backward(tc=True) needs."""
        self._train_tc = bool(tc)
        if tc:
            self._tc_pack()
        n, _, h, w = x.shape
        B = self._buffers(n, h, w)
        self._x = x
        L = self.levels
        inp, cin = x, self.in_ch
        for l in range(L):
            hl, wl, c = h >> l, w >> l, self.ch[l]
            self._conv(inp, cin * hl * wl, cin, B[f"a{l}"], c * hl * wl, c, n, hl, wl, 3, f"e{l}a", True)
            self._conv(B[f"a{l}"], c * hl * wl, c, B[f"e{l}"], c * hl * wl, c, n, hl, wl, 3, f"e{l}b", True)
            if l < L - 1:
                self._ok(self.lib.glbm_nn_pool2(_ptr(B[f"e{l}"]), c * hl * wl, _ptr(B[f"p{l}"]),
                                                c * hl * wl // 4, c, n, hl, wl, 0, 0, self._stream()), "pool")
                inp, cin = B[f"p{l}"], c
        top, ctop = B[f"e{L - 1}"], self.ch[L - 1]
        for l in range(L - 2, -1, -1):
            hl, wl, c = h >> l, w >> l, self.ch[l]
            cc = ctop + c
            cat = B[f"cat{l}"]
            self._ok(self.lib.glbm_nn_upsample2(_ptr(top), ctop * (hl // 2) * (wl // 2), _ptr(cat), cc * hl * wl,
                                                ctop, n, hl // 2, wl // 2, 0, self._stream()), "upsample")
            self._ok(self.lib.glbm_nn_copy_channels(_ptr(B[f"e{l}"]), c * hl * wl, _ptr(cat, ctop * hl * wl),
                                                    cc * hl * wl, c, n, hl, wl, 0, self._stream()), "copy")
            self._conv(cat, cc * hl * wl, cc, B[f"da{l}"], c * hl * wl, c, n, hl, wl, 3, f"d{l}a", True)
            self._conv(B[f"da{l}"], c * hl * wl, c, B[f"d{l}"], c * hl * wl, c, n, hl, wl, 3, f"d{l}b", True)
            top, ctop = B[f"d{l}"], c
        self._conv(top, ctop * h * w, ctop, B["y"], self.out_ch * h * w, self.out_ch, n, h, w, 1, "head", False)
        self._train_tc = False
        return B["y"]

    def backward(self, gy, tc=False):
        """Gradients of the loss w.r.t. the parameters (into self.grads) given
        gy = dL/dy of the last forward call (tc: on the tensor cores; the
        forward call must have used tc=True too)."""
        if tc and not self._xh:
            raise RuntimeError("backward(tc=True) needs a forward(tc=True) first")
        self._train_tc = bool(tc)
        if tc:
            self._tc_pack()
            self._tc_pack_flip()
        x = self._x
        n, _, h, w = x.shape
        B = self._buffers(n, h, w)
        L = self.levels
        self.grads.zero_()
        top = B["d0"] if L > 1 else B["e0"]
        gtop = B["gd0"] if L > 1 else B["ge0"]
        c0 = self.ch[0]
        self._conv_bwd(top, c0 * h * w, c0, gy, self.out_ch * h * w, self.out_ch, n, h, w, 1, "head",
                       dx=gtop, dxbs=c0 * h * w)
        for l in range(0, L - 1):
            hl, wl, c = h >> l, w >> l, self.ch[l]
            cup = self.ch[l + 1]
            cc = cup + c
            self._relu_bwd(B[f"d{l}"], B[f"gd{l}"], c, n, hl, wl)
            self._conv_bwd(B[f"da{l}"], c * hl * wl, c, B[f"gd{l}"], c * hl * wl, c, n, hl, wl, 3, f"d{l}b",
                           dx=B[f"gda{l}"], dxbs=c * hl * wl)
            self._relu_bwd(B[f"da{l}"], B[f"gda{l}"], c, n, hl, wl)
            self._conv_bwd(B[f"cat{l}"], cc * hl * wl, cc, B[f"gda{l}"], c * hl * wl, c, n, hl, wl, 3, f"d{l}a",
                           dx=B[f"gcat{l}"], dxbs=cc * hl * wl)
            gcat = B[f"gcat{l}"]
            self._ok(self.lib.glbm_nn_copy_channels(_ptr(gcat, cup * hl * wl), cc * hl * wl, _ptr(B[f"ge{l}"]),
                                                    c * hl * wl, c, n, hl, wl, 0, self._stream()), "copy")
            dst = B[f"ge{L - 1}"] if l + 1 == L - 1 else B[f"gd{l + 1}"]
            self._ok(self.lib.glbm_nn_upsample2(_ptr(gcat), cc * hl * wl, _ptr(dst), cup * (hl // 2) * (wl // 2),
                                                cup, n, hl // 2, wl // 2, 1, self._stream()), "upsample_bwd")
        for l in range(L - 1, -1, -1):
            hl, wl, c = h >> l, w >> l, self.ch[l]
            if l < L - 1:
                self._ok(self.lib.glbm_nn_pool2(_ptr(B[f"gp{l}"]), c * hl * wl // 4, _ptr(B[f"ge{l}"]),
                                                c * hl * wl, c, n, hl, wl, 1, 1, self._stream()), "pool_bwd")
            self._relu_bwd(B[f"e{l}"], B[f"ge{l}"], c, n, hl, wl)
            self._conv_bwd(B[f"a{l}"], c * hl * wl, c, B[f"ge{l}"], c * hl * wl, c, n, hl, wl, 3, f"e{l}b",
                           dx=B[f"ga{l}"], dxbs=c * hl * wl)
            self._relu_bwd(B[f"a{l}"], B[f"ga{l}"], c, n, hl, wl)
            if l == 0:
                self._conv_bwd(x, self.in_ch * h * w, self.in_ch, B["ga0"], c * h * w, c, n, h, w, 3, "e0a")
            else:
                cp = self.ch[l - 1]
                self._conv_bwd(B[f"p{l - 1}"], cp * hl * wl, cp, B[f"ga{l}"], c * hl * wl, c, n, hl, wl, 3,
                               f"e{l}a", dx=B[f"gp{l - 1}"], dxbs=cp * hl * wl)
        self._train_tc = False

    # -- tensor-core training ------------------------------------------------
    def _nhwc(self, store, key, src, c, n, h, w):
        """FP32 NCHW src (c channels) -> BF16 NHWC with max(32, c rounded up to
        32) channels, zero padded; kept in store[key]."""
        torch = self.torch
        cp = max(32, self._pad(c, 32))
        buf = store.get(key)
        if buf is None or tuple(buf.shape) != (n, h, w, cp):
            buf = torch.empty((n, h, w, cp), dtype=torch.bfloat16, device="cuda")
            store[key] = buf
        self._ok(self.lib.glbm_nn_nchw_to_nhwc(_ptr(src), n, c, h, w, C.c_void_p(buf.data_ptr()), cp,
                                               self._stream()), "nchw_to_nhwc")
        return buf, cp

    def _tc_err(self):
        torch = self.torch
        if getattr(self, "_tc_errbuf", None) is None:
            self._tc_errbuf = torch.zeros(1, dtype=torch.int32, device="cuda")
        return C.c_void_p(self._tc_errbuf.data_ptr())

    def _conv_tc(self, x, cin, y, cout, n, h, w, k, name, relu):
        xh, cp = self._nhwc(self._xh, name, x, cin, n, h, w)
        _, W, Bs = self._tc
        cop = Bs[name].numel()
        self._ok(self.lib.glbm_nn_tc_conv(
            C.c_void_p(xh.data_ptr()), cp, None, 0, n, h, w, k, C.c_void_p(W[name].data_ptr()),
            C.c_void_p(Bs[name].data_ptr()), cop, _ptr(y), cop, int(relu), 1, cout, self._tc_err(),
            self._stream()), "tc_conv")

    def _conv_bwd_tc(self, cin, dy, cout, n, h, w, k, name, dx):
        xh = self._xh[name]
        dyh, cyp = self._nhwc(self._gh, (n, h, w, cout), dy, cout, n, h, w)
        ow, ob = self._wb(name)
        self._ok(self.lib.glbm_nn_tc_conv_wgrad(C.c_void_p(xh.data_ptr()), xh.shape[3], cin,
                                                C.c_void_p(dyh.data_ptr()), cyp, cout, n, h, w, k,
                                                _ptr(self.grads, ow), self._tc_err(), self._stream()), "tc_wgrad")
        self._ok(self.lib.glbm_nn_bias_grad(_ptr(dy), cout * h * w, cout, n, h, w, _ptr(self.grads, ob),
                                            self._stream()), "bias_grad")
        if dx is not None:
            # the gradient convolution has cin outputs, run in groups of at
            # most 256 (the MMA's N); a group beyond the first writes a
            # scratch tensor that is copied into its channel slice of dx
            _, WF, ZB = self._tct
            for c0, cg, cgp, wt in WF[name]:
                out = dx if len(WF[name]) == 1 else self._dx_scratch(n, cg, h, w)
                self._ok(self.lib.glbm_nn_tc_conv(
                    C.c_void_p(dyh.data_ptr()), cyp, None, 0, n, h, w, k, C.c_void_p(wt.data_ptr()),
                    C.c_void_p(ZB[cgp].data_ptr()), cgp, _ptr(out), cgp, 0, 1, cg, self._tc_err(),
                    self._stream()), "tc_conv (input gradient)")
                if out is not dx:
                    self._ok(self.lib.glbm_nn_copy_channels(_ptr(out), cg * h * w, _ptr(dx, c0 * h * w), cin * h * w,
                                                            cg, n, h, w, 0, self._stream()), "copy")

    def _dx_scratch(self, n, c, h, w):
        torch = self.torch
        t = getattr(self, "_dxs", None)
        if t is None or t.numel() < n * c * h * w:
            t = self._dxs = torch.empty(n * c * h * w, dtype=torch.float32, device="cuda")
        return t

    def _tc_pack_flip(self):
        """BF16 weights of the input-gradient convolutions (flipped in space,
        input and output channels swapped), repacked when the parameters
        change."""
        if self._tct is not None and self._tct[0] == self._version:
            return self._tct
        torch = self.torch
        WF, ZB = {}, {}
        for name, ci, co, k in self.specs:
            cyp = max(32, self._pad(co, 32))      # input channels of the gradient convolution
            WF[name] = []
            for c0 in range(0, ci, 256):           # its outputs, in groups of <= 256
                cg = min(256, ci - c0)
                cgp = max(16, self._pad(cg, 16))
                wt = torch.empty(k * k * cgp * cyp, dtype=torch.bfloat16, device="cuda")
                ow, _ = self._wb(name)
                self._ok(self.lib.glbm_nn_tc_pack_weights_flip(_ptr(self.params, ow), co, ci, k, c0, cgp, cyp,
                                                               C.c_void_p(wt.data_ptr()), self._stream()),
                         "pack_flip")
                WF[name].append((c0, cg, cgp, wt))
                if cgp not in ZB:
                    ZB[cgp] = torch.zeros(cgp, dtype=torch.float32, device="cuda")
        self._tct = (self._version, WF, ZB)
        return self._tct

    def loss(self, pred, target, channel_weight, with_grad=True):
        torch = self.torch
        n, c, h, w = pred.shape
        cw = torch.as_tensor(channel_weight, dtype=torch.float32, device="cuda")
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.empty_like(pred) if with_grad else None
        self._ok(self.lib.glbm_nn_mse(_ptr(pred), _ptr(target), _ptr(cw), c, n, h, w,
                                      _ptr(g) if g is not None else None, C.c_void_p(out.data_ptr()),
                                      self._stream()), "mse")
        return out, g

    def coarse_loss(self, pred, target, factor, weight, grad):
        """Adds weight * mean((pool^k pred_0 - pool^k target_0)^2), k = log2(factor),
        of the first channel to the loss, and its gradient to grad (channel 0).
        Emphasises the large-scale density field that the slow pressure modes
        carry.  Returns the device loss."""
        torch = self.torch
        n, c, h, w = pred.shape
        steps = int(round(np.log2(factor)))
        p_prev, t_prev, ps, ts = pred, target, [], []
        hh, ww, sb = h, w, c * h * w
        for _ in range(steps):
            p_new = torch.empty((n, 1, hh // 2, ww // 2), dtype=torch.float32, device="cuda")
            t_new = torch.empty_like(p_new)
            for src, dst in ((p_prev, p_new), (t_prev, t_new)):
                self._ok(self.lib.glbm_nn_pool2(_ptr(src), sb, _ptr(dst), hh * ww // 4, 1, n, hh, ww, 0, 0,
                                                self._stream()), "pool")
            ps.append((p_new, hh, ww))
            p_prev, t_prev, sb = p_new, t_new, hh * ww // 4
            hh, ww = hh // 2, ww // 2
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        cw = torch.tensor([weight], dtype=torch.float32, device="cuda")
        g = torch.empty_like(p_prev)
        self._ok(self.lib.glbm_nn_mse(_ptr(p_prev), _ptr(t_prev), _ptr(cw), 1, n, hh, ww, _ptr(g),
                                      C.c_void_p(loss.data_ptr()), self._stream()), "mse")
        # back through the pools; the last one accumulates into grad[:, 0]
        for k in range(steps - 1, -1, -1):
            _, h_in, w_in = ps[k]
            if k == 0:
                self._ok(self.lib.glbm_nn_pool2(_ptr(g), h_in * w_in // 4, _ptr(grad), c * h_in * w_in, 1, n,
                                                h_in, w_in, 1, 1, self._stream()), "pool_bwd")
            else:
                g_up = torch.empty((n, 1, h_in, w_in), dtype=torch.float32, device="cuda")
                self._ok(self.lib.glbm_nn_pool2(_ptr(g), h_in * w_in // 4, _ptr(g_up), h_in * w_in, 1, n, h_in,
                                                w_in, 1, 0, self._stream()), "pool_bwd")
                g = g_up
        return loss

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        self._version += 1
        self._ok(self.lib.glbm_nn_adam(_ptr(self.params), _ptr(self.grads), _ptr(self.m), _ptr(self.v),
                                       self.nparams, float(lr), float(beta1), float(beta2), float(eps), self.t,
                                       self._stream()), "adam")

    def save(self, path, half=False):
        """Parameters as .npy (FP16 when half: the network still computes in
        FP32; the rounding is far below the prediction error)."""
        p = self.params.cpu().numpy()
        np.save(path, p.astype(np.float16) if half else p)

    def load(self, path):
        p = np.load(path).astype(np.float32)
        if p.size != self.nparams:
            raise ValueError(f"{path}: {p.size} parameters, this network has {self.nparams}")
        self.params.copy_(self.torch.from_numpy(p).cuda())
        self._version += 1

    def invalidate_tc(self):
        """Call after writing ``params`` directly: the tensor-core path
        repacks its BF16 weights on the next ``forward_tc``."""
        self._version += 1

    # -- tensor-core inference ------------------------------------------------
    @staticmethod
    def _pad(c, m):
        return (c + m - 1) // m * m

    def _tc_pack(self):
        if self._tc is not None and self._tc[0] == self._version:
            return self._tc
        torch = self.torch
        W, Bs = {}, {}
        for name, ci, co, k in self.specs:
            cip = max(32, self._pad(ci, 32))
            cop = self._pad(co, 16)
            wt = torch.empty(k * k * cop * cip, dtype=torch.bfloat16, device="cuda")
            ow, ob = self._wb(name)
            self._ok(self.lib.glbm_nn_tc_pack_weights(_ptr(self.params, ow), co, ci, k, cop, cip,
                                                      C.c_void_p(wt.data_ptr()), self._stream()), "tc_pack")
            b = torch.zeros(cop, dtype=torch.float32, device="cuda")
            b[:co] = self.params[ob:ob + co]
            W[name], Bs[name] = wt, b
            if name == "e0a" and k == 3 and ci <= 16:
                # inference reads the network input padded to 16 channels, not 32
                w16 = torch.empty(9 * cop * 16, dtype=torch.bfloat16, device="cuda")
                self._ok(self.lib.glbm_nn_tc_pack_weights(_ptr(self.params, ow), co, ci, 3, cop, 16,
                                                          C.c_void_p(w16.data_ptr()), self._stream()), "tc_pack")
                W["e0a_c16"] = w16
            if name == "e0a" and k == 3 and 9 * ci <= 32:
                # the same weights [co][ci][3][3] read as a 1x1 convolution of the
                # 3x3 patches (glbm_nn_im2col3_nhwc): [co][9 ci][1][1]
                wi = torch.empty(cop * 32, dtype=torch.bfloat16, device="cuda")
                self._ok(self.lib.glbm_nn_tc_pack_weights(_ptr(self.params, ow), co, 9 * ci, 1, cop, 32,
                                                          C.c_void_p(wi.data_ptr()), self._stream()), "tc_pack")
                W["e0a_im2col"] = wi
        self._tc = (self._version, W, Bs)
        return self._tc

    def _tc_buffers(self, n, h, w):
        key = (n, h, w)
        if key in self._tc_bufs:
            return self._tc_bufs[key]
        if h % 2 ** (self.levels - 1) or w % 2 ** (self.levels - 1):
            raise ValueError(f"h, w must be multiples of {2 ** (self.levels - 1)}")
        torch = self.torch

        def z(c, l):
            return torch.empty((n, h >> l, w >> l, c), dtype=torch.bfloat16, device="cuda")
        B = {"x": z(max(32, self._pad(self.in_ch, 32), self._pad(9 * self.in_ch, 32) if 9 * self.in_ch <= 32 else 0), 0)}
        if self.in_ch <= 16:
            B["x16"] = z(16, 0)
        L = self.levels
        for l in range(L):
            c = self.ch[l]
            B[f"a{l}"], B[f"e{l}"] = z(c, l), z(c, l)
            if l < L - 1:
                B[f"p{l}"] = z(c, l + 1)
                B[f"u{l}"] = z(self.ch[l + 1], l)
                B[f"da{l}"], B[f"d{l}"] = z(c, l), z(c, l)
        B["y"] = torch.empty((n, self.out_ch, h, w), dtype=torch.float32, device="cuda")
        B["err"] = torch.zeros(1, dtype=torch.int32, device="cuda")
        self._tc_bufs = {key: B}
        return B

    def _tc_conv(self, B, x0, c0, x1, c1, n, h, w, name, relu, y, head=False, wkey=None, k=None):
        _, W, Bs = self._tc
        if k is None:
            k = 1 if head else 3
        cop = Bs[name].numel()
        self._ok(self.lib.glbm_nn_tc_conv(
            C.c_void_p(x0.data_ptr()), c0, C.c_void_p(x1.data_ptr()) if x1 is not None else None, c1,
            n, h, w, k, C.c_void_p(W[wkey or name].data_ptr()), C.c_void_p(Bs[name].data_ptr()), cop,
            C.c_void_p(y.data_ptr()), cop, int(relu), int(head), self.out_ch if head else 0,
            C.c_void_p(B["err"].data_ptr()), self._stream()), "tc_conv")

    def forward_tc(self, x, fused=True, im2col=False):
        """The forward pass on the tensor cores: x (n, in_ch, h, w) FP32 CUDA
        tensor -> (n, out_ch, h, w) FP32.  Activations are BF16 NHWC between
        layers, accumulation FP32; the pipeline's error flag is checked.
        fused: each level's 2x2 pooling runs inside the epilogue of the
        convolution before it where that layer takes the band kernel (32 or
        64 channels, rows of >= 128 pixels), a decoder level's 2x upsampling
        inside the epilogue of the convolution that makes its input where
        the streaming kernel takes that layer (glbm_nn_tc_conv_up2), and with
        a 32-channel first level the 1x1 head runs inside the last
        convolution's epilogue (glbm_nn_tc_conv_fused).
        im2col: with at most 3 input channels the first convolution runs as a
        1x1 convolution of the 3x3 patches (glbm_nn_im2col3_nhwc), 27 useful
        channels of 32 instead of 3 of 32 in each of 9 taps (off by default:
        at 2048^2 the patch tensor and the 1x1 tile convolution took 275 us
        against 210 us for the padded input and the streaming 3x3 kernel)."""
        n, _, h, w = x.shape
        self._tc_pack()
        B = self._tc_buffers(n, h, w)
        st = self._stream()
        _, W, _ = self._tc
        use_i2c = im2col and "e0a_im2col" in W
        use16 = not use_i2c and "e0a_c16" in W
        inp = B["x16"] if use16 else B["x"]
        cin = inp.shape[3]
        conv = self.lib.glbm_nn_im2col3_nhwc if use_i2c else self.lib.glbm_nn_nchw_to_nhwc
        self._ok(conv(_ptr(x), n, self.in_ch, h, w, C.c_void_p(inp.data_ptr()), cin, st),
                 "im2col3_nhwc" if use_i2c else "nchw_to_nhwc")
        L = self.levels
        fuse_head = fused and self.ch[0] == 32 and w >= 128

        def fuse_pool(l):
            c = self.ch[l]
            return (fused and l < L - 1 and c in (32, 64) and (w >> l) >= 128
                    and 9 * c * c * 2 <= 80 * 1024)

        for l in range(L):
            hl, wl, c = h >> l, w >> l, self.ch[l]
            if l == 0 and use_i2c:
                self._tc_conv(B, inp, cin, None, 0, n, hl, wl, "e0a", True, B["a0"], wkey="e0a_im2col", k=1)
            elif l == 0 and use16:
                self._tc_conv(B, inp, cin, None, 0, n, hl, wl, "e0a", True, B["a0"], wkey="e0a_c16")
            else:
                self._tc_conv(B, inp, cin, None, 0, n, hl, wl, f"e{l}a", True, B[f"a{l}"])
            if fuse_pool(l):
                self._tc_fused(B, B[f"a{l}"], c, n, hl, wl, f"e{l}b", c, y=B[f"e{l}"], pool_y=B[f"p{l}"])
            else:
                self._tc_conv(B, B[f"a{l}"], c, None, 0, n, hl, wl, f"e{l}b", True, B[f"e{l}"])
                if l < L - 1:
                    self._ok(self.lib.glbm_nn_pool2_nhwc(C.c_void_p(B[f"e{l}"].data_ptr()), n, c, hl, wl,
                                                         C.c_void_p(B[f"p{l}"].data_ptr()), st), "pool2_nhwc")
            if l < L - 1:
                inp, cin = B[f"p{l}"], c
        top, ctop = B[f"e{L - 1}"], self.ch[L - 1]
        upsampled = False  # the previous convolution wrote u{l} itself
        for l in range(L - 2, -1, -1):
            hl, wl, c = h >> l, w >> l, self.ch[l]
            if not upsampled:
                self._ok(self.lib.glbm_nn_upsample2_nhwc(C.c_void_p(top.data_ptr()), n, ctop, hl // 2, wl // 2,
                                                         C.c_void_p(B[f"u{l}"].data_ptr()), st), "upsample2_nhwc")
            self._tc_conv(B, B[f"u{l}"], ctop, B[f"e{l}"], c, n, hl, wl, f"d{l}a", True, B[f"da{l}"])
            if l == 0 and fuse_head:
                # d0b with the 1x1 head in its epilogue: d0 itself is never stored
                self._tc_fused(B, B["da0"], c, n, hl, wl, "d0b", c, head=True)
                return B["y"]
            upsampled = False
            if fused and l > 0 and c in (32, 64):
                # d{l}b writes the next level's upsampled input directly, where the
                # streaming kernel takes the layer (otherwise EINVAL: do it apart)
                _, W, Bs = self._tc
                rc = self.lib.glbm_nn_tc_conv_up2(
                    C.c_void_p(B[f"da{l}"].data_ptr()), c, None, 0, n, hl, wl, C.c_void_p(W[f"d{l}b"].data_ptr()),
                    C.c_void_p(Bs[f"d{l}b"].data_ptr()), c, C.c_void_p(B[f"u{l - 1}"].data_ptr()), c, 1,
                    C.c_void_p(B["err"].data_ptr()), st)
                if rc == 0:
                    upsampled = True
                elif rc != -1:
                    self._ok(rc, "tc_conv_up2")
            if not upsampled:
                self._tc_conv(B, B[f"da{l}"], c, None, 0, n, hl, wl, f"d{l}b", True, B[f"d{l}"])
            top, ctop = B[f"d{l}"], c
        self._tc_conv(B, top, ctop, None, 0, n, h, w, "head", False, B["y"], head=True)
        return B["y"]

    def _tc_fused(self, B, x0, c0, n, h, w, name, cout, y=None, pool_y=None, head=False):
        _, W, Bs = self._tc
        vp = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        self._ok(self.lib.glbm_nn_tc_conv_fused(
            vp(x0), c0, None, 0, n, h, w, vp(W[name]), vp(Bs[name]), cout, vp(y), cout, 1, vp(pool_y),
            vp(W["head"]) if head else None, vp(Bs["head"]) if head else None, self.out_ch if head else 0,
            vp(B["y"]) if head else None, vp(B["err"]), self._stream()), "tc_conv_fused")

    def flops(self, h, w, n=1):
        """Multiply-add work of one forward pass, 2 * pixels * cin * cout * k^2
        summed over the convolutions (real channel counts, no padding)."""
        level = {}
        for l in range(self.levels):
            level[f"e{l}a"] = level[f"e{l}b"] = l
            level[f"d{l}a"] = level[f"d{l}b"] = l
        level["head"] = 0
        return sum(2.0 * n * (h >> level[nm]) * (w >> level[nm]) * ci * co * k * k for nm, ci, co, k in self.specs)

    def tc_error(self):
        """Nonzero if a tensor-core pipeline wait timed out since the buffers
        were made, in inference or training (synchronises)."""
        for B in self._tc_bufs.values():
            if int(B["err"].item()):
                return int(B["err"].item())
        if getattr(self, "_tc_errbuf", None) is not None:
            return int(self._tc_errbuf.item())
        return 0


# -- data --------------------------------------------------------------------

def features(eps, K, G):
    """Network input (3, ny, nx) float32 from one medium."""
    f = np.empty((3,) + eps.shape, dtype=np.float32)
    f[0] = (eps - 0.05) / 0.05
    f[1] = (np.log10(K) + 2.0) / 2.0
    f[2] = np.log10(abs(G)) + 6.0
    return f


def targets(rho, ux, uy, K, G, nu):
    t = np.empty((3,) + rho.shape, dtype=np.float32)
    t[0] = (rho - 1.0) / (G * RHO_SCALE)
    t[1] = ux * nu / (K * G)
    t[2] = uy * nu / (K * G)
    return t


def predict_device(net, eps, K, G, nu, tc=True):
    """Warm-start fields from FP64 CUDA tensors eps, K (ny, nx), computed on
    the device end to end: features kernel, the network (tensor cores when
    tc, else the FP32 kernels), decode kernel.  Returns FP64 CUDA tensors
    (rho, ux, uy) for Solver.init_equilibrium."""
    torch = net.torch
    ny, nx = eps.shape
    npix = ny * nx
    st = net._stream()
    x = torch.empty((1, 3, ny, nx), dtype=torch.float32, device="cuda")
    net._ok(net.lib.glbm_nn_warm_features(_ptr(eps), _ptr(K), npix, float(G), _ptr(x), st), "warm_features")
    y = net.forward_tc(x) if tc else net.forward(x)
    out = [torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3)]
    net._ok(net.lib.glbm_nn_warm_decode(_ptr(y), _ptr(K), npix, float(G), float(nu), RHO_SCALE,
                                        *[_ptr(o) for o in out], st), "warm_decode")
    return tuple(out)


def decode(y, K, G, nu):
    """Network output (3, ny, nx) -> (rho, ux, uy) FP64."""
    y = np.asarray(y, dtype=np.float64)
    gs, g_nu = G * RHO_SCALE, G / nu
    return 1.0 + y[0] * gs, y[1] * K * g_nu, y[2] * K * g_nu
