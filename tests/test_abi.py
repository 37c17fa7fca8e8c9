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


def test_no_oracle_in_product():
    """The product package never imports the oracle (it is test-only)."""
    pkgdir = os.path.join(ROOT, "paper_1601_00704_gb300")
    for dp, _, files in os.walk(pkgdir):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                src = open(os.path.join(dp, f)).read()
                assert "oracle" not in src.lower().replace("oracle-", ""), f
