"""Tensor-core (tcgen05) inference kernels of the warm-start network against
the FP64 NumPy oracle (convolution on the same BF16-rounded inputs and
weights) and against the FP32 network kernels (whole U-Net), through the C
ABI.  BF16 NHWC activations, FP32 accumulation."""

import ctypes as C

import numpy as np
import pytest

from oracle import unet as ou

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1601_00704_gb300 import build
    build.build()
    import paper_1601_00704_gb300 as p
    p.load()
    return p


def _bf16(a):
    """Round to BF16 (nearest even) and back, on the host."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _vp(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# (n, h, w, c0, c1, cout, ksize, relu, f32 head output)
CASES = [
    (1, 16, 16, 32, 0, 32, 3, True, False),     # 2-D tile 16 x 8
    (2, 20, 24, 64, 32, 48, 3, False, False),   # width not dividing 128, two input tensors
    (1, 9, 200, 32, 0, 16, 3, True, False),     # wider than a tile, ragged in x and y
    (1, 8, 8, 128, 128, 128, 3, True, False),   # smaller than one tile (rows beyond the image)
    (2, 32, 40, 32, 0, 16, 1, False, True),     # 1x1 head, FP32 NCHW output of 3 channels
    (1, 64, 256, 64, 0, 64, 3, True, False),    # several full 128-pixel tiles per row
    (2, 5, 130, 64, 32, 48, 3, False, False),   # one-row tiles, two input tensors, a 2-pixel last tile
    (1, 3, 384, 128, 128, 128, 3, True, False), # one-row tiles at the widest channel counts
    # band kernel shapes (3x3, rows >= 128 pixels, cout <= 64):
    (1, 17, 256, 64, 32, 32, 3, True, False),   # two input tensors, 3 chunks, ragged last band (8 + 8 + 1 rows)
    (2, 16, 128, 32, 0, 32, 3, True, False),    # one pixel tile per row, two images
    (1, 12, 300, 32, 32, 64, 3, False, False),  # 4-row bands, a 44-pixel last tile
    (1, 8, 2048, 32, 0, 32, 3, True, False),    # one band of 8 rows across 16 pixel tiles
    (1, 640, 128, 32, 0, 32, 3, True, False),   # 160 bands: CTAs reuse both accumulator buffers (stacked)
    (1, 640, 128, 32, 0, 64, 3, False, False),  # 160 bands, 64 output channels (unstacked)
    # a first layer with 16 input channels (the loads zero-fill the chunk's other 16):
    (2, 20, 40, 16, 0, 32, 3, True, False),     # tile kernel
    (1, 24, 256, 16, 0, 32, 3, True, False),    # band / streaming
    (1, 12, 300, 16, 0, 64, 3, True, False),    # band, 64 output channels
    (1, 12, 256, 128, 64, 64, 3, True, False),  # 221 KB of weights: tile kernel, or streaming with the weights in each stage
]


@pytest.mark.parametrize("variant", [1, 0, 3, 2, 5])
@pytest.mark.parametrize("n,h,w,c0,c1,cout,k,relu,head", CASES)
def test_tc_conv_matches_oracle(pkg, n, h, w, c0, c1, cout, k, relu, head, variant):
    """Every case on the tile kernel (variant 1), with the per-layer choice
    (variant 0: the band kernel wherever it applies, with the dy taps
    stacked along N for 32 output channels), with the band kernel
    unstacked (variant 3), with the tile kernel's ring never deepened
    (variant 2; in the other variants grids of at most one CTA per SM, most
    of the small cases here, take the 8-stage ring, which the 72 K steps of
    the 256-channel case wrap nine times) and with the streaming form of the
    32-channel band layers however short its segments (variant 5)."""
    import torch
    lib = pkg.load()
    lib.glbm_nn_tc_set_variant(variant)
    rng = np.random.default_rng(hash((n, h, w, c0, c1, cout, k)) % 2 ** 32)
    cin = c0 + c1
    x = _bf16(rng.normal(size=(n, cin, h, w)))
    wf = rng.normal(0.0, np.sqrt(2.0 / (cin * k * k)), size=(cout, cin, k, k)).astype(np.float32)
    b = rng.normal(0.0, 0.1, size=cout).astype(np.float32)
    ref = ou.conv(x, _bf16(wf), b.astype(np.float64))
    if relu:
        ref = np.maximum(ref, 0.0)

    nhwc = torch.from_numpy(x.transpose(0, 2, 3, 1).astype(np.float32)).to(torch.bfloat16).cuda()
    x0 = nhwc[..., :c0].contiguous()
    x1 = nhwc[..., c0:].contiguous() if c1 else None
    wt = torch.empty(k * k * cout * cin, dtype=torch.bfloat16, device="cuda")
    wdev = torch.from_numpy(wf.ravel()).cuda()
    assert lib.glbm_nn_tc_pack_weights(_vp(wdev), cout, cin, k, cout, cin, _vp(wt), _stream()) == 0
    bdev = torch.from_numpy(b).cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    store = 3 if head else 0
    if head:
        y = torch.full((n, store, h, w), float("nan"), dtype=torch.float32, device="cuda")
    else:
        y = torch.full((n, h, w, cout), float("nan"), dtype=torch.bfloat16, device="cuda")
    rc = lib.glbm_nn_tc_conv(_vp(x0), c0, _vp(x1) if x1 is not None else None, c1, n, h, w, k, _vp(wt),
                             _vp(bdev), cout, _vp(y), cout, int(relu), int(head), store, _vp(err), _stream())
    lib.glbm_nn_tc_set_variant(0)
    assert rc == 0, pkg.load().glbm_last_error(None)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    scale = np.abs(ref).max()
    if head:
        got = y.cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got, ref[:, :store], rtol=0, atol=2e-6 * scale)
    else:
        got = y.float().cpu().numpy().astype(np.float64).transpose(0, 3, 1, 2)
        assert np.isfinite(got).all()
        # the BF16 output rounding (half an ulp = 2^-9 relative) plus FP32 accumulation
        bound = 2.0 ** -8 * np.abs(ref) + 1e-6 * scale
        assert (np.abs(got - ref) <= bound).all(), np.abs(got - ref).max()


def _band_layer(pkg, rng, n, h, w, c0, c1, variant, fused, cout=32):
    """One 3x3 layer with 32 or 64 output channels and ReLU under the given
    kernel variant: (output, pooled output or None, head output or None;
    the fused head only with 32 output channels)."""
    import torch
    lib = pkg.load()
    cin = c0 + c1
    nhwc = torch.from_numpy(rng.normal(size=(n, h, w, cin)).astype(np.float32)).to(torch.bfloat16).cuda()
    x0 = nhwc[..., :c0].contiguous()
    x1 = nhwc[..., c0:].contiguous() if c1 else None
    wf = rng.normal(0.0, np.sqrt(2.0 / (cin * 9)), size=(cout, cin, 3, 3)).astype(np.float32)
    wt = torch.empty(9 * cout * cin, dtype=torch.bfloat16, device="cuda")
    assert lib.glbm_nn_tc_pack_weights(_vp(torch.from_numpy(wf.ravel()).cuda()), cout, cin, 3, cout, cin,
                                       _vp(wt), _stream()) == 0
    bdev = torch.from_numpy(rng.normal(0.0, 0.1, size=cout).astype(np.float32)).cuda()
    hw = torch.from_numpy(rng.normal(0.0, 0.2, size=3 * 32).astype(np.float32)).to(torch.bfloat16).cuda()
    hb = torch.from_numpy(rng.normal(0.0, 0.1, size=3).astype(np.float32)).cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = torch.full((n, h, w, cout), float("nan"), dtype=torch.bfloat16, device="cuda")
    pool = head = None
    lib.glbm_nn_tc_set_variant(variant)
    try:
        if fused:
            pool = torch.full((n, h // 2, w // 2, cout), float("nan"), dtype=torch.bfloat16, device="cuda")
            if cout == 32:
                head = torch.full((n, 3, h, w), float("nan"), dtype=torch.float32, device="cuda")
            rc = lib.glbm_nn_tc_conv_fused(_vp(x0), c0, _vp(x1) if x1 is not None else None, c1, n, h, w, _vp(wt),
                                           _vp(bdev), cout, _vp(y), cout, 1, _vp(pool),
                                           _vp(hw) if head is not None else None,
                                           _vp(hb) if head is not None else None, 3 if head is not None else 0,
                                           _vp(head) if head is not None else None, _vp(err), _stream())
        else:
            rc = lib.glbm_nn_tc_conv(_vp(x0), c0, _vp(x1) if x1 is not None else None, c1, n, h, w, 3, _vp(wt),
                                     _vp(bdev), cout, _vp(y), cout, 1, 0, 0, _vp(err), _stream())
    finally:
        lib.glbm_nn_tc_set_variant(0)
    assert rc == 0, lib.glbm_last_error(None)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return y, pool, head


@pytest.mark.parametrize("n,h,w,c0,c1,fused,cout", [
    (150, 40, 128, 32, 0, True, 32),    # one 40-row segment per image: 42 input rows wrap the 16-slot ring
    (100, 34, 128, 64, 32, False, 32),  # three chunks from two tensors
    (70, 35, 200, 32, 0, False, 32),    # odd rows (a half-used last pair), a 72-pixel last strip
    (1, 300, 2048, 32, 0, True, 32),    # 16 strips x 9 segments of 34 rows (the last 28)
    (100, 34, 128, 16, 0, False, 32),   # a 16-channel input: two blocks and one K step per tap
    (150, 40, 128, 32, 0, True, 64),    # 64 output channels: the 8-slot ring wrapped five times, fused pooling
    (76, 33, 200, 64, 0, False, 64),    # two chunks, odd rows, ragged last strip
    (1, 300, 1024, 32, 32, True, 64),   # two tensors, 8 strips x 19 segments
    (76, 33, 200, 128, 64, False, 64),  # weights too large to keep: each stage brings its chunk's 9 tiles
    (1, 300, 1024, 96, 0, False, 64),   # the same, one tensor of 3 chunks, 8 strips x 19 segments
])
def test_streaming_conv_matches_band_kernel(pkg, n, h, w, c0, c1, fused, cout):
    """The streaming form (variant 5) against the band kernel (variant 4,
    stacked for 32 output channels; the tile kernel where the weights exceed
    the band kernel's 80 KB), on layers whose segments wrap the TMEM
    row ring: the same products of the same BF16 values, summed in the same
    order for one 32-channel chunk and in another chunk order for two or
    three, so outputs agree to at most one BF16 ulp (exactly for one chunk,
    but for rounding differences the tensor core may make between an MMA
    and the same MMA split at the ring's wrap); fused pooling and head
    likewise."""
    import torch
    seed = n * 1000 + h + cout
    y4, p4, h4 = _band_layer(pkg, np.random.default_rng(seed), n, h, w, c0, c1, 4, fused, cout)
    y5, p5, h5 = _band_layer(pkg, np.random.default_rng(seed), n, h, w, c0, c1, 5, fused, cout)
    # relative bound: one BF16 ulp (<= 2^-7) for the outputs; a pooled value
    # averages four outputs that may each be one ulp off (ReLU: all >= 0, so
    # at most 2^-7 of the average) and is rounded again: 2^-6
    pairs = [(y4.float(), y5.float(), 2.0 ** -7)]
    if fused:
        pairs.append((p4.float(), p5.float(), 2.0 ** -6))
    if h4 is not None:
        pairs.append((h4, h5, 2.0 ** -7))
    for a, b, rel in pairs:
        assert torch.isfinite(b).all()
        d = (a - b).abs()
        assert float((d - rel * a.abs()).max()) <= 1e-6 * float(a.abs().max()), float(d.max())
        if c1 == 0 and c0 <= 32:
            same = float((d == 0).float().mean())
            print(f"exactly equal: {same:.6f}")
            assert same > 0.999


@pytest.mark.parametrize("n,h,w,c0,c1,cout,extra", [
    (2, 20, 136, 32, 0, 32, 0),    # 32 channels, a 8-pixel last strip
    (1, 34, 256, 64, 0, 64, 0),    # 64 channels, two chunks
    (3, 17, 200, 32, 32, 64, 16),  # two tensors, odd rows, written into a 80-channel tensor's first 64
])
def test_conv_up2_matches_conv_then_upsample(pkg, n, h, w, c0, c1, cout, extra):
    """glbm_nn_tc_conv_up2 (the streaming kernel writing its output 2x
    nearest-upsampled by TMA stores) gives, bit for bit, the plain streaming
    convolution followed by glbm_nn_upsample2_nhwc, and leaves the channels
    beyond cout of a wider output tensor alone."""
    import torch
    lib = pkg.load()
    rng = np.random.default_rng(n * 100 + h + cout)
    cin = c0 + c1
    nhwc = torch.from_numpy(rng.normal(size=(n, h, w, cin)).astype(np.float32)).to(torch.bfloat16).cuda()
    x0 = nhwc[..., :c0].contiguous()
    x1 = nhwc[..., c0:].contiguous() if c1 else None
    wf = rng.normal(0.0, np.sqrt(2.0 / (cin * 9)), size=(cout, cin, 3, 3)).astype(np.float32)
    wt = torch.empty(9 * cout * cin, dtype=torch.bfloat16, device="cuda")
    assert lib.glbm_nn_tc_pack_weights(_vp(torch.from_numpy(wf.ravel()).cuda()), cout, cin, 3, cout, cin,
                                       _vp(wt), _stream()) == 0
    bdev = torch.from_numpy(rng.normal(0.0, 0.1, size=cout).astype(np.float32)).cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    xp1 = _vp(x1) if x1 is not None else None
    lib.glbm_nn_tc_set_variant(5)
    try:
        y = torch.empty((n, h, w, cout), dtype=torch.bfloat16, device="cuda")
        assert lib.glbm_nn_tc_conv(_vp(x0), c0, xp1, c1, n, h, w, 3, _vp(wt), _vp(bdev), cout, _vp(y), cout, 1, 0, 0,
                                   _vp(err), _stream()) == 0
        ref = torch.empty((n, 2 * h, 2 * w, cout), dtype=torch.bfloat16, device="cuda")
        assert lib.glbm_nn_upsample2_nhwc(_vp(y), n, cout, h, w, _vp(ref), _stream()) == 0
        ys = cout + extra
        up = torch.full((n, 2 * h, 2 * w, ys), float("nan"), dtype=torch.bfloat16, device="cuda")
        rc = lib.glbm_nn_tc_conv_up2(_vp(x0), c0, xp1, c1, n, h, w, _vp(wt), _vp(bdev), cout, _vp(up), ys, 1,
                                     _vp(err), _stream())
    finally:
        lib.glbm_nn_tc_set_variant(0)
    assert rc == 0, lib.glbm_last_error(None)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert torch.equal(up[..., :cout], ref)
    if extra:
        assert torch.isnan(up[..., cout:].float()).all()


def test_conv_up2_needs_the_streaming_kernel(pkg):
    import torch
    lib = pkg.load()
    buf = torch.zeros(1 << 16, dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(32, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    # rows of 64 pixels: no 128-pixel strip
    assert lib.glbm_nn_tc_conv_up2(_vp(buf), 32, None, 0, 1, 8, 64, _vp(buf), _vp(b), 32, _vp(buf), 32, 1,
                                   _vp(err), _stream()) == -1
    assert b"streaming" in lib.glbm_last_error(None)
    # 48 output channels
    assert lib.glbm_nn_tc_conv_up2(_vp(buf), 32, None, 0, 1, 8, 256, _vp(buf), _vp(b), 48, _vp(buf), 48, 1,
                                   _vp(err), _stream()) == -1


def test_tc_conv_rejects_bad_shapes(pkg):
    import torch
    lib = pkg.load()
    buf = torch.zeros(4096, dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(64, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")

    def call(c0, cout, k):
        return lib.glbm_nn_tc_conv(_vp(buf), c0, None, 0, 1, 4, 4, k, _vp(buf), _vp(b), cout, _vp(buf), cout,
                                   1, 0, 0, _vp(err), _stream())
    assert call(40, 32, 3) == -1   # input channels not a multiple of 16
    assert b"multiples of 32" in lib.glbm_last_error(None)
    assert lib.glbm_nn_tc_conv(_vp(buf), 16, _vp(buf), 32, 1, 4, 4, 3, _vp(buf), _vp(b), 32, _vp(buf), 32,
                               1, 0, 0, _vp(err), _stream()) == -1  # 16 + 32: chunks would straddle the tensors
    assert call(32, 24, 3) == -1   # cout not a multiple of 16
    assert b"cout" in lib.glbm_last_error(None)
    assert call(32, 32, 5) == -1   # kernel size 5
    assert b"k = 1 or 3" in lib.glbm_last_error(None)


@pytest.mark.parametrize("n,c,h,w,cp", [(1, 90, 9, 37, 96), (2, 3, 4, 4, 264), (3, 128, 8, 8, 128),
                                         (1, 32, 64, 64, 32)],
                         ids=["ragged-run", "two-slices", "small", "aligned"])
def test_nchw_to_nhwc_matches_torch(pkg, n, c, h, w, cp):
    """FP32 NCHW -> BF16 NHWC (zero-padded to cp channels) bit for bit against
    torch's round-to-nearest-even conversion: a run of pixels shorter than 32
    at the end of each image, more than 256 channels (two slices of the
    shared-memory tile), small and aligned tensors."""
    import torch
    lib = pkg.load()
    rng = np.random.default_rng(c * 1000 + h * w)
    x = rng.normal(size=(n, c, h, w)).astype(np.float32)
    y = torch.full((n, h, w, cp), 7.0, dtype=torch.bfloat16, device="cuda")
    assert lib.glbm_nn_nchw_to_nhwc(_vp(torch.from_numpy(x).cuda()), n, c, h, w, _vp(y), cp, _stream()) == 0
    expect = np.zeros((n, h, w, cp), dtype=np.float32)
    expect[..., :c] = x.transpose(0, 2, 3, 1)
    torch.cuda.synchronize()
    assert torch.equal(y.cpu(), torch.from_numpy(expect).to(torch.bfloat16))


def test_nhwc_layout_kernels(pkg):
    import torch
    lib = pkg.load()
    rng = np.random.default_rng(5)
    n, c, h, w = 2, 5, 6, 10
    x = rng.normal(size=(n, c, h, w)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty((n, h, w, 16), dtype=torch.bfloat16, device="cuda")
    assert lib.glbm_nn_nchw_to_nhwc(_vp(xd), n, c, h, w, _vp(y), 16, _stream()) == 0
    expect = np.zeros((n, h, w, 16), dtype=np.float32)
    expect[..., :c] = x.transpose(0, 2, 3, 1)
    exp_bf = torch.from_numpy(expect).to(torch.bfloat16)
    assert torch.equal(y.cpu(), exp_bf)

    # pool: FP32 sum (a + b) + (d + e), times 1/4, rounded to BF16
    pooled = torch.empty((n, h // 2, w // 2, 16), dtype=torch.bfloat16, device="cuda")
    assert lib.glbm_nn_pool2_nhwc(_vp(y), n, 16, h, w, _vp(pooled), _stream()) == 0
    v = exp_bf.float().numpy()
    s = (v[:, 0::2, 0::2] + v[:, 0::2, 1::2]) + (v[:, 1::2, 0::2] + v[:, 1::2, 1::2])
    ref = torch.from_numpy((np.float32(0.25) * s).astype(np.float32)).to(torch.bfloat16)
    assert torch.equal(pooled.cpu(), ref)

    up = torch.empty((n, h, w, 16), dtype=torch.bfloat16, device="cuda")
    assert lib.glbm_nn_upsample2_nhwc(_vp(pooled), n, 16, h // 2, w // 2, _vp(up), _stream()) == 0
    ref_up = ref.repeat_interleave(2, dim=1).repeat_interleave(2, dim=2)
    assert torch.equal(up.cpu(), ref_up)


def test_im2col3_layout(pkg):
    """3x3 patches as channels, bit for bit: channel ci * 9 + 3 (dy + 1) +
    (dx + 1) holds x[ci][y + dy][x + dx], zero outside the image and in the
    padding channels."""
    import torch
    lib = pkg.load()
    rng = np.random.default_rng(6)
    n, c, h, w = 2, 3, 7, 11
    x = rng.normal(size=(n, c, h, w)).astype(np.float32)
    y = torch.full((n, h, w, 32), float("nan"), dtype=torch.bfloat16, device="cuda")
    assert lib.glbm_nn_im2col3_nhwc(_vp(torch.from_numpy(x).cuda()), n, c, h, w, _vp(y), 32, _stream()) == 0
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    expect = np.zeros((n, h, w, 32), dtype=np.float32)
    for ci in range(c):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                expect[..., ci * 9 + 3 * (dy + 1) + (dx + 1)] = xp[:, ci, 1 + dy:1 + dy + h, 1 + dx:1 + dx + w]
    assert torch.equal(y.cpu(), torch.from_numpy(expect).to(torch.bfloat16))
    assert lib.glbm_nn_im2col3_nhwc(_vp(torch.from_numpy(x).cuda()), n, 4, h, w, _vp(y), 32, _stream()) == -1


@pytest.mark.parametrize("n,h,w,cin", [(2, 40, 136, 3), (1, 9, 64, 2)])
def test_first_layer_as_patch_convolution_matches_oracle(pkg, n, h, w, cin):
    """A 3x3 convolution of a few input channels computed as the 1x1
    tensor-core convolution of its 3x3 patches, with the FP32 weights
    [cout][cin][3][3] packed as [cout][9 cin][1][1], against the oracle's
    3x3 convolution on the same BF16-rounded inputs and weights."""
    import torch
    lib = pkg.load()
    rng = np.random.default_rng(31 + cin)
    cout = 32
    x = rng.normal(size=(n, cin, h, w)).astype(np.float32)
    wf = rng.normal(0.0, np.sqrt(2.0 / (cin * 9)), size=(cout, cin, 3, 3)).astype(np.float32)
    b = rng.normal(0.0, 0.1, size=cout).astype(np.float32)
    ref = np.maximum(ou.conv(_bf16(x), _bf16(wf), b.astype(np.float64)), 0.0)
    patches = torch.empty((n, h, w, 32), dtype=torch.bfloat16, device="cuda")
    assert lib.glbm_nn_im2col3_nhwc(_vp(torch.from_numpy(x).cuda()), n, cin, h, w, _vp(patches), 32,
                                    _stream()) == 0
    wt = torch.empty(cout * 32, dtype=torch.bfloat16, device="cuda")
    assert lib.glbm_nn_tc_pack_weights(_vp(torch.from_numpy(wf.ravel()).cuda()), cout, 9 * cin, 1, cout, 32,
                                       _vp(wt), _stream()) == 0
    y = torch.full((n, h, w, cout), float("nan"), dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.glbm_nn_tc_conv(_vp(patches), 32, None, 0, n, h, w, 1, _vp(wt), _vp(torch.from_numpy(b).cuda()),
                               cout, _vp(y), cout, 1, 0, 0, _vp(err), _stream()) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = y.float().cpu().numpy().astype(np.float64).transpose(0, 3, 1, 2)
    bound = 2.0 ** -8 * np.abs(ref) + 1e-6 * np.abs(ref).max()
    assert (np.abs(got - ref) <= bound).all(), np.abs(got - ref).max()


@pytest.mark.parametrize("h,w,c0,c1", [(16, 256, 64, 0), (6, 384, 32, 32)])
def test_fused_pool_64_channels_matches_separate_kernels(pkg, h, w, c0, c1):
    """The band kernel with 64 output channels and the 2x2 pooling in its
    epilogue writes what the plain band convolution followed by
    glbm_nn_pool2_nhwc writes, bit for bit (the same FP32 arithmetic on the
    same BF16 values); a fused head needs 32 output channels."""
    import torch
    lib = pkg.load()
    rng = np.random.default_rng(h * w + c1)
    n, cout, cin = 2, 64, c0 + c1
    nhwc = torch.from_numpy(rng.normal(size=(n, h, w, cin)).astype(np.float32)).to(torch.bfloat16).cuda()
    x0 = nhwc[..., :c0].contiguous()
    x1 = nhwc[..., c0:].contiguous() if c1 else None
    wf = rng.normal(0.0, np.sqrt(2.0 / (cin * 9)), size=(cout, cin, 3, 3)).astype(np.float32)
    wt = torch.empty(9 * cout * cin, dtype=torch.bfloat16, device="cuda")
    assert lib.glbm_nn_tc_pack_weights(_vp(torch.from_numpy(wf.ravel()).cuda()), cout, cin, 3, cout, cin,
                                       _vp(wt), _stream()) == 0
    bdev = torch.from_numpy(rng.normal(0.0, 0.1, size=cout).astype(np.float32)).cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    xp1 = _vp(x1) if x1 is not None else None
    y0 = torch.empty((n, h, w, cout), dtype=torch.bfloat16, device="cuda")
    assert lib.glbm_nn_tc_conv(_vp(x0), c0, xp1, c1, n, h, w, 3, _vp(wt), _vp(bdev), cout, _vp(y0), cout, 1, 0, 0,
                               _vp(err), _stream()) == 0
    p0 = torch.empty((n, h // 2, w // 2, cout), dtype=torch.bfloat16, device="cuda")
    assert lib.glbm_nn_pool2_nhwc(_vp(y0), n, cout, h, w, _vp(p0), _stream()) == 0
    y1 = torch.full_like(y0, float("nan"))
    p1 = torch.full_like(p0, float("nan"))
    assert lib.glbm_nn_tc_conv_fused(_vp(x0), c0, xp1, c1, n, h, w, _vp(wt), _vp(bdev), cout, _vp(y1), cout, 1,
                                     _vp(p1), None, None, 0, None, _vp(err), _stream()) == 0, \
        lib.glbm_last_error(None)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert torch.equal(y0, y1)
    assert torch.equal(p0, p1)
    hw = torch.zeros(4 * 32, dtype=torch.bfloat16, device="cuda")
    hy = torch.zeros((n, 1, h, w), dtype=torch.float32, device="cuda")
    assert lib.glbm_nn_tc_conv_fused(_vp(x0), c0, xp1, c1, n, h, w, _vp(wt), _vp(bdev), cout, _vp(y1), cout, 1,
                                     None, _vp(hw), _vp(bdev), 1, _vp(hy), _vp(err), _stream()) == -1
    assert b"32 output channels" in lib.glbm_last_error(None)


@pytest.mark.parametrize("levels,max_ch,size", [(3, 64, 32), (4, None, 64), (3, 64, 256)])
def test_unet_forward_tc_matches_fp32(pkg, levels, max_ch, size):
    """Random-initialised network: the tensor-core forward pass agrees with the
    FP32 kernels to the BF16 activation rounding accumulated over the layers."""
    import torch
    from paper_1601_00704_gb300.surrogate import UNet
    net = UNet(base=32, levels=levels, seed=3, max_ch=max_ch)
    rng = np.random.default_rng(11)
    x = torch.from_numpy(rng.normal(size=(2, 3, size, size)).astype(np.float32)).cuda()
    y32 = net.forward(x).clone()
    ytc = net.forward_tc(x).clone()
    torch.cuda.synchronize()
    assert net.tc_error() == 0
    rel = float((ytc - y32).norm() / y32.norm())
    assert rel < 2e-2, rel


@pytest.mark.parametrize("levels,size", [(3, 256), (6, 512)])
def test_unet_forward_tc_fused_matches_unfused(pkg, levels, size):
    """The fused levels (2x2 pooling inside the band kernel's epilogue at
    the 32- and 64-channel levels, the 1x1 head inside the last
    convolution's) give what the separate kernels give: the pooled tensors
    exactly (same arithmetic on the same BF16 values), the network output
    to FP32 summation order."""
    import torch
    from paper_1601_00704_gb300.surrogate import UNet
    net = UNet(base=32, levels=levels, seed=7, max_ch=128)
    rng = np.random.default_rng(17)
    x = torch.from_numpy(rng.normal(size=(2, 3, size, size)).astype(np.float32)).cuda()
    key = (2, size, size)
    y0 = net.forward_tc(x, fused=False, im2col=False).clone()
    p0 = [net._tc_bufs[key][f"p{l}"].clone() for l in (0, 1)]
    y1 = net.forward_tc(x, fused=True, im2col=False).clone()
    p1 = [net._tc_bufs[key][f"p{l}"].clone() for l in (0, 1)]
    torch.cuda.synchronize()
    assert net.tc_error() == 0
    for a, b in zip(p0, p1):
        assert torch.equal(a, b)
    rel = float((y1 - y0).abs().max() / y0.abs().max())
    assert rel < 1e-5, rel


def test_unet_forward_tc_first_layer_as_patches(pkg):
    """The first convolution as the 1x1 convolution of 3x3 patches sums the
    same BF16 products in another order: its output agrees with the direct
    3x3 form to about one BF16 ulp, and the network output to well below
    the BF16 activation error of the pass."""
    import torch
    from paper_1601_00704_gb300.surrogate import UNet
    net = UNet(base=32, levels=4, seed=9, max_ch=128)
    rng = np.random.default_rng(19)
    x = torch.from_numpy(rng.normal(size=(1, 3, 256, 256)).astype(np.float32)).cuda()
    key = (1, 256, 256)
    y0 = net.forward_tc(x, im2col=False).clone()
    a0 = net._tc_bufs[key]["a0"].float().clone()
    y1 = net.forward_tc(x, im2col=True).clone()
    a1 = net._tc_bufs[key]["a0"].float().clone()
    torch.cuda.synchronize()
    assert net.tc_error() == 0
    assert float((a1 - a0).abs().max()) <= 2.0 ** -7 * float(a0.abs().max())
    rel = float((y1 - y0).norm() / y0.norm())
    assert rel < 1e-2, rel


def test_trained_network_tc_prediction(pkg):
    """The committed network on an unseen medium of its training recipe: the
    tensor-core prediction matches the FP32 one in every output channel."""
    import json
    import os

    import torch

    import media
    from paper_1601_00704_gb300 import surrogate
    from paper_1601_00704_gb300 import train_surrogate as T
    meta = json.load(open(os.path.splitext(T.DEFAULT_WEIGHTS)[0] + ".json"))
    net = surrogate.UNet(base=meta["base"], levels=meta["levels"], max_ch=meta.get("max_ch"))
    net.load(T.DEFAULT_WEIGHTS)
    m = media.shale_batch(1, seed=9101, sides=(256,))[0]
    K = T.medium_k(pkg, m)
    x = torch.from_numpy(surrogate.features(m["eps"], K, T.G)[None]).cuda()
    y32 = net.forward(x).clone()
    ytc = net.forward_tc(x).clone()
    torch.cuda.synchronize()
    assert net.tc_error() == 0
    for ch in range(3):
        rel = float((ytc[0, ch] - y32[0, ch]).norm() / y32[0, ch].norm())
        print(f"channel {ch}: relative L2 difference {rel:.2e}")
        assert rel < 3e-2, (ch, rel)


def test_device_features_and_decode_match_host(pkg):
    """The device-resident warm-start plumbing computes what the host
    definitions (surrogate.features / decode) compute: decode bit for bit,
    features within a few FP32 roundings (the kernel works in FP32 on the
    rounded eps and K, the host in FP64)."""
    import torch

    import media
    from paper_1601_00704_gb300 import surrogate
    from paper_1601_00704_gb300 import train_surrogate as T
    lib = pkg.load()
    m = media.shale_batch(1, seed=9102, sides=(64,))[0]
    K = T.medium_k(pkg, m)
    eps_d = torch.from_numpy(np.ascontiguousarray(m["eps"], dtype=np.float64)).cuda()
    K_d = torch.from_numpy(np.ascontiguousarray(K, dtype=np.float64)).cuda()
    x = torch.empty((3, 64, 64), dtype=torch.float32, device="cuda")
    assert lib.glbm_nn_warm_features(_vp(eps_d), _vp(K_d), 64 * 64, T.G, _vp(x), _stream()) == 0
    ref = surrogate.features(m["eps"], K, T.G)
    got = x.cpu().numpy()
    # |feature| <= ~3: a few ulps of FP32 at that magnitude
    np.testing.assert_allclose(got[:2], ref[:2], rtol=0, atol=2e-6)
    np.testing.assert_allclose(got[2], ref[2], rtol=0, atol=1e-9)  # log10|G| + 6, host libm on both sides

    y = np.random.default_rng(3).normal(size=(3, 64, 64)).astype(np.float32)
    yd = torch.from_numpy(y).cuda()
    out = [torch.empty((64, 64), dtype=torch.float64, device="cuda") for _ in range(3)]
    assert lib.glbm_nn_warm_decode(_vp(yd), _vp(K_d), 64 * 64, T.G, T.NU, surrogate.RHO_SCALE,
                                   *[_vp(o) for o in out], _stream()) == 0
    for got, exp in zip(out, surrogate.decode(y, K, T.G, T.NU)):
        assert np.array_equal(got.cpu().numpy(), exp)
