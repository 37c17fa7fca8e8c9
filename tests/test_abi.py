"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every entry point include/glbm.h declares."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(glbm_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1601_00704_gb300 import build
    build.build()
    import paper_1601_00704_gb300 as pkg
    return pkg.load()


def test_exports_every_declared_symbol(lib):
    names = declared("glbm.h")
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_1601_00704_gb300 as pkg
    assert sorted(pkg.SYMBOLS) == declared("glbm.h")


def test_create_error_message_without_device(lib):
    """Argument checks happen before any CUDA call: a bad size is rejected
    with EINVAL and a message, even on a host without a GPU."""
    import ctypes as C
    h = C.c_void_p()
    rc = lib.glbm_create(1, 8, 1.0, 0, 0, None, C.byref(h))
    assert rc == -1 and h.value is None
    assert b"nx, ny >= 2" in lib.glbm_last_error(None)
    rc = lib.glbm_create(8, 8, 0.4, 0, 0, None, C.byref(h))
    assert rc == -1 and b"tau" in lib.glbm_last_error(None)
    lib.glbm_destroy(None)  # NULL-safe


def test_elementwise_entry_points_reject_empty_images(lib):
    """Sizes are checked on the host before any CUDA call (so this runs
    without a GPU; the placeholder pointers are never dereferenced):
    images without pixels, and odd sizes for 2x2 pooling, are EINVAL."""
    import ctypes as C
    p = C.c_void_p(256)
    assert lib.glbm_nn_relu_bwd(p, 0, p, 0, 3, 2, 0, 8, None) == -1
    assert lib.glbm_nn_copy_channels(p, 0, p, 0, 3, 2, 8, 0, 0, None) == -1
    for h, w in ((0, 8), (8, 0), (1, 8), (7, 8)):
        assert lib.glbm_nn_pool2(p, 0, p, 0, 3, 2, h, w, 0, 0, None) == -1
    assert lib.glbm_nn_upsample2(p, 0, p, 0, 3, 2, 0, 4, 0, None) == -1


def test_tensor_core_entry_points_validate_on_the_host(lib):
    """The weight gradient and the layout conversion reject bad sizes and
    misaligned pointers with EINVAL and a message before any CUDA call."""
    import ctypes as C
    p, q = C.c_void_p(256), C.c_void_p(256 + 4)

    def wgrad(x=p, cx=32, cin=32, cy=32, cout=32, k=3):
        return lib.glbm_nn_tc_conv_wgrad(x, cx, cin, p, cy, cout, 2, 8, 8, k, p, p, None)

    assert wgrad(k=5) == -1 and b"k = 1 or 3" in lib.glbm_last_error(None)
    assert wgrad(cx=48) == -1 and b"multiples of 32" in lib.glbm_last_error(None)
    assert wgrad(cy=288, cout=288) == -1
    assert wgrad(cin=40) == -1      # more real input channels than the tensor holds
    assert wgrad(x=q) == -1 and b"16-byte aligned" in lib.glbm_last_error(None)
    assert lib.glbm_nn_nchw_to_nhwc(p, 2, 5, 4, 4, p, 12, None) == -1     # c_pad not a multiple of 8
    assert lib.glbm_nn_nchw_to_nhwc(p, 2, 20, 4, 4, p, 16, None) == -1    # c_pad < c
    assert lib.glbm_nn_nchw_to_nhwc(p, 2, 5, 4, 4, q, 16, None) == -1     # y not 16-byte aligned
    assert b"16-byte aligned" in lib.glbm_last_error(None)


def test_no_oracle_in_product():
    """The product package never imports the oracle (it is test-only)."""
    pkgdir = os.path.join(ROOT, "paper_1601_00704_gb300")
    for dp, _, files in os.walk(pkgdir):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                src = open(os.path.join(dp, f)).read()
                assert "oracle" not in src.lower().replace("oracle-", ""), f
