"""The allocation-free step entry point, glbm_step_reduce_noalloc.

Some callers may not allocate device memory themselves: applications whose
host framework owns the whole device-memory budget and hands out every
buffer, or pipelines that must not risk the implicit device synchronisation
of cudaMalloc/cudaFree mid-loop.  For them the library offers one step that
runs on caller-owned buffers, with the reduction scratch in a fixed array
compiled into the library.  These tests call it through the C ABI and check
it against the ordinary handle-based glbm_step on two calls in a row, with
the FP32 step tolerances of the parity suite (|df| <= 1e-6 * n * max|g|,
|dU| <= 2e-5 * n * max|U|).

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""

import ctypes as C

import numpy as np
import pytest

import media

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.fixture(scope="module")
def env():
    from paper_1601_00704_gb300 import build
    build.build()
    import torch

    import paper_1601_00704_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return pkg, pkg.load(), torch


def ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


@pytest.mark.parametrize("nx,ny,walls,forch", [(256, 64, True, False),
                                               (250, 40, False, True)])
def test_noalloc_matches_glbm_step_twice(env, nx, ny, walls, forch):
    pkg, lib, torch = env
    tau, gx, gy = 0.9, 2e-5, -5e-6
    eps, K = media.random_medium(nx, ny, seed=nx + ny, k_range=(1e-3, 1e0))
    nu = (tau - 0.5) / 3
    N = nx * ny
    plane = (N + 63) // 64 * 64
    feps = 0.8 if forch else 0.0
    # caller-owned device buffers: state at rest (zero deviations) and the
    # per-node coefficients eps*nu/K, eps (and eps*F_eps/sqrt(K))
    bufs = [torch.zeros(9 * plane, dtype=torch.float32, device="cuda") for _ in range(2)]
    alpha = torch.from_numpy((eps * nu / K).astype(np.float32)).cuda()
    epsf = torch.from_numpy(eps.astype(np.float32)).cuda()
    beta = torch.from_numpy((eps * feps / np.sqrt(K)).astype(np.float32)).cuda() if forch else None
    mean = torch.zeros(2, dtype=torch.float64, device="cuda")

    ref = pkg.Solver(nx, ny, tau=tau, walls=walls)
    ref.set_medium(eps, K, feps)
    ref.set_force(gx, gy)
    flags = 0 if walls else 1
    for call in (1, 2):
        src, dst = bufs[(call - 1) % 2], bufs[call % 2]
        rc = lib.glbm_step_reduce_noalloc(ptr(src), ptr(dst), ptr(alpha), ptr(epsf), ptr(beta),
                                          nx, ny, plane, tau, gx, gy, flags, ptr(mean), None)
        assert rc == 0, lib.glbm_last_error(None).decode()
        torch.cuda.synchronize()
        ref.step(1)
        want_f = ref.distributions()
        want_u = ref.mean_velocity()
        got_f = dst.view(9, plane)[:, :N].double().cpu().numpy().reshape(9, ny, nx) + W[:, None, None]
        got_u = mean.cpu().numpy()
        gmax = np.abs(want_f - W[:, None, None]).max()
        np.testing.assert_allclose(got_f, want_f, rtol=0, atol=1e-6 * call * gmax)
        np.testing.assert_allclose(got_u, want_u, rtol=0, atol=2e-5 * call * np.abs(want_u).max())


def test_noalloc_rejects_oversize_lattice(env):
    """Beyond the fixed scratch (65536 reduction blocks) the call fails with
    EINVAL before touching any buffer."""
    pkg, lib, torch = env
    nx, ny = 4096, 8193  # 8 blocks per row * 8193 rows > 65536
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    mean = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = lib.glbm_step_reduce_noalloc(ptr(buf), ptr(buf[32:]), ptr(buf), ptr(buf), None,
                                      nx, ny, nx * ny, 1.0, 1e-6, 0.0, 0, ptr(mean), None)
    assert rc == -1
    assert b"fixed scratch" in lib.glbm_last_error(None)


def test_noalloc_rejects_overlapping_buffers(env):
    """A destination that overlaps a buffer the step reads (here g_dst
    starting inside g_src, or mean_u inside alpha) is refused with EINVAL
    before anything is enqueued."""
    pkg, lib, torch = env
    nx, ny = 64, 8
    plane = nx * ny
    f = torch.zeros(2 * 9 * plane, dtype=torch.float32, device="cuda")
    coef = torch.ones(2 * plane, dtype=torch.float32, device="cuda")
    mean = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = lib.glbm_step_reduce_noalloc(ptr(f), ptr(f[9 * plane - 64:]), ptr(coef), ptr(coef[plane:]), None,
                                      nx, ny, plane, 1.0, 1e-6, 0.0, 0, ptr(mean), None)
    assert rc == -1 and b"overlaps" in lib.glbm_last_error(None)
    rc = lib.glbm_step_reduce_noalloc(ptr(f), ptr(f[9 * plane:]), ptr(coef), ptr(coef[plane:]), None,
                                      nx, ny, plane, 1.0, 1e-6, 0.0, 0, ptr(coef[4:]), None)
    assert rc == -1 and b"overlaps" in lib.glbm_last_error(None)
    # disjoint buffers are accepted
    rc = lib.glbm_step_reduce_noalloc(ptr(f), ptr(f[9 * plane:]), ptr(coef), ptr(coef[plane:]), None,
                                      nx, ny, plane, 1.0, 1e-6, 0.0, 0, ptr(mean), None)
    assert rc == 0, lib.glbm_last_error(None).decode()
    torch.cuda.synchronize()


def test_noalloc_allocates_no_device_memory(env):
    """After the first call (which looks up the scratch array's address), a
    run of further calls leaves the device's free memory and the caching
    allocator's reservation unchanged."""
    pkg, lib, torch = env
    nx, ny = 512, 256
    plane = nx * ny
    f = torch.zeros(2 * 9 * plane, dtype=torch.float32, device="cuda")
    coef = torch.full((2 * plane,), 0.5, dtype=torch.float32, device="cuda")
    mean = torch.zeros(2, dtype=torch.float64, device="cuda")
    halves = (f[:9 * plane], f[9 * plane:])

    def call(k):
        rc = lib.glbm_step_reduce_noalloc(ptr(halves[k % 2]), ptr(halves[(k + 1) % 2]), ptr(coef),
                                          ptr(coef[plane:]), None, nx, ny, plane, 1.0, 1e-6, 0.0, 0,
                                          ptr(mean), None)
        assert rc == 0, lib.glbm_last_error(None).decode()

    call(0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for k in range(1, 21):
        call(k)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0
    assert torch.cuda.memory_reserved() == reserved0
    assert np.isfinite(mean.cpu().numpy()).all()
