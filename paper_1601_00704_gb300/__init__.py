"""GB300-native generalized lattice Boltzmann model (GLBM) for gas flow in
voxelised organic shale (Wang, Chen, Kang & Rahman, arXiv:1601.00704, Sec. 2.3).

Every lattice node carries its own porosity eps and apparent permeability K;
the time loop (Eqs. 27-37) runs as hand-written CUDA kernels for sm_103a in
``libglbm.so`` behind the C ABI of ``include/glbm.h``.  This package is the
thin Python binding over that ABI: it marshals arguments (NumPy host arrays
or CUDA torch tensors) and raises on error codes.  There is no CPU or
PyTorch fallback: importing works anywhere, but creating a ``Solver`` needs
the built library and a CUDA device, and fails loudly otherwise.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB as LIB_PATH

__all__ = ["Solver", "Batch", "kapp_field", "em_gmm1d", "GLBMError", "load", "F32", "F64",
           "F16DEV", "BF16DEV", "WALLS_Y", "PERIODIC_Y", "NEAREST16", "STORAGE"]

F32, F64, F16DEV, BF16DEV = 0, 1, 2, 3
STORAGE = {"f32": F32, "f64": F64, "f16": F16DEV, "bf16": BF16DEV}
WALLS_Y, PERIODIC_Y, NEAREST16 = 0, 1, 2

_STATUS = {0: "GLBM_OK", -1: "GLBM_EINVAL", -2: "GLBM_ENOMEM",
           -3: "GLBM_ECUDA", -4: "GLBM_ENAN", -5: "GLBM_ESTATE"}

# Symbols the header declares (checked by the CPU test-suite).
SYMBOLS = ["glbm_create", "glbm_set_medium", "glbm_set_force",
           "glbm_init_equilibrium", "glbm_step", "glbm_mean_velocity",
           "glbm_permeability", "glbm_get_velocity", "glbm_get_distributions",
           "glbm_counters", "glbm_destroy", "glbm_last_error",
           "glbm_step_reduce_noalloc", "glbm_debug_fail_launch", "glbm_debug_guards",
           "glbm_batch_debug_guards", "glbm_save", "glbm_load",
           "glbm_set_convergence", "glbm_batch_set_persistent", "glbm_batch_get_persistent",
           "glbm_batch_set_convergence", "glbm_nn_tc_set_variant",
           "glbm_nn_tc_conv_wgrad", "glbm_nn_tc_pack_weights_flip", "glbm_nn_bias_grad",
           "glbm_nn_tc_conv_fused",
           "glbm_batch_create", "glbm_batch_set_medium", "glbm_batch_set_force",
           "glbm_batch_reset", "glbm_batch_set_schedule", "glbm_batch_autotune",
           "glbm_batch_step", "glbm_batch_results", "glbm_batch_get_distributions",
           "glbm_batch_info", "glbm_batch_destroy", "glbm_batch_last_error",
           "glbm_kapp_field", "glbm_qsat_from_langmuir_volume",
           "glbm_batch_get_fields",
           "glbm_nn_conv_fwd", "glbm_nn_conv_bwd_data", "glbm_nn_conv_bwd_weight",
           "glbm_nn_relu_bwd", "glbm_nn_copy_channels", "glbm_nn_pool2",
           "glbm_nn_upsample2", "glbm_nn_mse", "glbm_nn_adam", "glbm_em_gmm1d",
           "glbm_nn_tc_conv", "glbm_nn_tc_pack_weights", "glbm_nn_nchw_to_nhwc", "glbm_nn_im2col3_nhwc",
           "glbm_nn_tc_debug_starve", "glbm_nn_tc_conv_up2",
           "glbm_nn_pool2_nhwc", "glbm_nn_upsample2_nhwc", "glbm_nn_warm_features",
           "glbm_nn_warm_decode"]


class GLBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = _STATUS.get(code, str(code))


_lib = None
_PD = C.POINTER(C.c_double)
_VP = C.c_void_p


def load(path: str | None = None) -> C.CDLL:
    """Load libglbm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libglbm.so not built at {p}; run "
                          "paper_1601_00704_gb300.build.build() first")
    lib = C.CDLL(p)
    i, ll, d, h = C.c_int, C.c_longlong, C.c_double, _VP
    sig = {
        "glbm_create": ([i, i, d, i, C.c_uint, _VP, C.POINTER(_VP)], i),
        "glbm_set_medium": ([h, _VP, _VP, d, i], i),
        "glbm_set_force": ([h, d, d], i),
        "glbm_init_equilibrium": ([h, _VP, _VP, _VP, i], i),
        "glbm_step": ([h, ll, d, i, C.POINTER(ll), C.POINTER(i)], i),
        "glbm_mean_velocity": ([h, _PD], i),
        "glbm_permeability": ([h, _PD], i),
        "glbm_get_velocity": ([h, _VP, _VP, i], i),
        "glbm_get_distributions": ([h, _VP, i], i),
        "glbm_counters": ([h, C.POINTER(ll), C.POINTER(ll)], i),
        "glbm_destroy": ([h], None),
        "glbm_debug_fail_launch": ([ll], None),
        "glbm_debug_guards": ([h, i, C.POINTER(ll)], i),
        "glbm_batch_debug_guards": ([h, i, C.POINTER(ll)], i),
        "glbm_save": ([h, C.c_char_p], i),
        "glbm_set_convergence": ([h, i], i),
        "glbm_batch_set_persistent": ([h, i], i),
        "glbm_batch_set_convergence": ([h, i], i),
        "glbm_nn_tc_set_variant": ([i], None),
        "glbm_nn_tc_debug_starve": ([i], None),
        "glbm_nn_tc_conv_up2": ([_VP, i, _VP, i, i, i, i, _VP, _VP, i, _VP, ll, i, _VP, _VP], i),
        "glbm_nn_tc_conv_wgrad": ([_VP, i, i, _VP, i, i, i, i, i, i, _VP, _VP, _VP], i),
        "glbm_nn_tc_pack_weights_flip": ([_VP, i, i, i, i, i, i, _VP, _VP], i),
        "glbm_nn_bias_grad": ([_VP, ll, i, i, i, i, _VP, _VP], i),
        "glbm_nn_tc_conv_fused": ([_VP, i, _VP, i, i, i, i, _VP, _VP, i, _VP, ll, i, _VP, _VP, _VP, i, _VP,
                                   _VP, _VP], i),
        "glbm_batch_get_persistent": ([h, C.POINTER(i)], i),
        "glbm_load": ([h, C.c_char_p], i),
        "glbm_last_error": ([h], C.c_char_p),
        "glbm_step_reduce_noalloc": ([_VP, _VP, _VP, _VP, _VP, i, i, ll, d, d, d,
                                      C.c_uint, _VP, _VP], i),
        "glbm_batch_create": ([i, _VP, _VP, d, i, C.c_uint, _VP, C.POINTER(_VP)], i),
        "glbm_batch_set_medium": ([h, i, _VP, _VP, i], i),
        "glbm_batch_set_force": ([h, d, d], i),
        "glbm_batch_reset": ([h], i),
        "glbm_batch_set_schedule": ([h, i, i], i),
        "glbm_batch_autotune": ([h, i, C.POINTER(i), C.POINTER(i)], i),
        "glbm_batch_step": ([h, ll, d, i, C.POINTER(ll), C.POINTER(i)], i),
        "glbm_batch_results": ([h, _VP, _VP, _VP, _VP], i),
        "glbm_batch_get_distributions": ([h, i, _VP, i], i),
        "glbm_batch_info": ([h, C.POINTER(i), C.POINTER(i), C.POINTER(ll), C.POINTER(ll)], i),
        "glbm_batch_destroy": ([h], None),
        "glbm_batch_last_error": ([h], C.c_char_p),
        "glbm_kapp_field": ([_VP, _VP, _VP, ll, d, d, d, d, d, d, d, d, d, _VP, i, _VP], i),
        "glbm_qsat_from_langmuir_volume": ([d] * 6, d),
        "glbm_batch_get_fields": ([h, i, _VP, _VP, _VP, i], i),
        "glbm_nn_conv_fwd": ([_VP, ll, i, _VP, ll, i, i, i, i, i, _VP, _VP, i, _VP], i),
        "glbm_nn_conv_bwd_data": ([_VP, ll, i, _VP, ll, i, i, i, i, i, _VP, _VP, _VP], i),
        "glbm_nn_conv_bwd_weight": ([_VP, ll, i, _VP, ll, i, i, i, i, i, _VP, _VP, _VP], i),
        "glbm_nn_relu_bwd": ([_VP, ll, _VP, ll, i, i, i, i, _VP], i),
        "glbm_nn_copy_channels": ([_VP, ll, _VP, ll, i, i, i, i, i, _VP], i),
        "glbm_nn_pool2": ([_VP, ll, _VP, ll, i, i, i, i, i, i, _VP], i),
        "glbm_nn_upsample2": ([_VP, ll, _VP, ll, i, i, i, i, i, _VP], i),
        "glbm_nn_mse": ([_VP, _VP, _VP, i, i, i, i, _VP, _VP, _VP], i),
        "glbm_nn_adam": ([_VP, _VP, _VP, _VP, ll, C.c_float, C.c_float, C.c_float,
                          C.c_float, i, _VP], i),
        "glbm_em_gmm1d": ([_VP, ll, i, _PD, _PD, _PD, i, d, C.POINTER(i), _PD, i, _VP], i),
        "glbm_nn_tc_conv": ([_VP, i, _VP, i, i, i, i, i, _VP, _VP, i, _VP, ll, i, i, i, _VP, _VP], i),
        "glbm_nn_tc_pack_weights": ([_VP, i, i, i, i, i, _VP, _VP], i),
        "glbm_nn_nchw_to_nhwc": ([_VP, i, i, i, i, _VP, i, _VP], i),
        "glbm_nn_im2col3_nhwc": ([_VP, i, i, i, i, _VP, i, _VP], i),
        "glbm_nn_pool2_nhwc": ([_VP, i, i, i, i, _VP, _VP], i),
        "glbm_nn_upsample2_nhwc": ([_VP, i, i, i, i, _VP, _VP], i),
        "glbm_nn_warm_features": ([_VP, _VP, ll, d, _VP, _VP], i),
        "glbm_nn_warm_decode": ([_VP, _VP, ll, d, d, d, _VP, _VP, _VP, _VP], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path is None:
        _lib = lib
    return lib


def _is_tensor(a) -> bool:
    return type(a).__module__.startswith("torch")


class _Arg:
    """Marshal one FP64 [ny][nx] (or [9][ny][nx]) array: NumPy on the host or
    a contiguous CUDA torch tensor on the device."""

    def __init__(self, a, shape, writable=False):
        self.obj = None
        self.device = False
        if a is None:
            self.ptr = None
            return
        if _is_tensor(a):
            import torch
            if a.dtype != torch.float64 or tuple(a.shape) != shape:
                raise ValueError(f"expected float64 tensor of shape {shape}")
            if not a.is_cuda:
                a = a.numpy()
            else:
                if not a.is_contiguous():
                    if writable:
                        raise ValueError("output tensor must be contiguous")
                    a = a.contiguous()
                self.obj, self.ptr, self.device = a, a.data_ptr(), True
                return
        if writable:
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64
                    and a.shape == shape and a.flags.c_contiguous):
                raise ValueError(f"output must be a C-contiguous float64 array {shape}")
            arr = a
        else:
            arr = np.ascontiguousarray(a, dtype=np.float64)
            if arr.shape != shape:
                raise ValueError(f"expected shape {shape}, got {arr.shape}")
        self.obj, self.ptr = arr, arr.ctypes.data


class Solver:
    """One GLBM lattice on the current CUDA device (a ``glbm_t`` handle).

    ``storage`` is 'f32' (default), 'f64', 'f16' or 'bf16'; ``walls`` puts
    halfway bounce-back walls at y = -1/2 and ny - 1/2 (else periodic y);
    ``stream`` is a ``torch.cuda.Stream`` (or raw cudaStream_t int), default
    the legacy default stream; ``flags`` adds further ``glbm_create`` flags
    (``NEAREST16``).
    """

    def __init__(self, nx, ny, tau=1.0, storage="f32", walls=True, stream=None,
                 flags=0):
        self._lib = load()
        self._h = _VP()
        self.nx, self.ny, self.tau = int(nx), int(ny), float(tau)
        st = STORAGE[storage] if isinstance(storage, str) else int(storage)
        s = stream
        if s is not None and not isinstance(s, int):
            s = s.cuda_stream
        self._stream = s
        rc = self._lib.glbm_create(self.nx, self.ny, self.tau, st,
                                   (WALLS_Y if walls else PERIODIC_Y) | int(flags),
                                   _VP(s) if s else None, C.byref(self._h))
        if rc != 0:
            raise GLBMError(rc, self._lib.glbm_last_error(None).decode())
        self.storage = storage
        self.gx = self.gy = 0.0

    # -- plumbing ----------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise GLBMError(rc, self._lib.glbm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.glbm_destroy(self._h)
            self._h = _VP()

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def shape(self):
        return (self.ny, self.nx)

    @property
    def nu(self):
        return (self.tau - 0.5) / 3.0

    # -- API ---------------------------------------------------------------
    def set_medium(self, eps, K, F_eps=0.0):
        e = _Arg(eps, self.shape)
        k = _Arg(K, self.shape)
        if e.device != k.device:
            raise ValueError("eps and K must both be host or both device arrays")
        self._check(self._lib.glbm_set_medium(self._h, e.ptr, k.ptr,
                                              float(F_eps), int(e.device)))

    def set_force(self, gx, gy=0.0):
        self._check(self._lib.glbm_set_force(self._h, float(gx), float(gy)))
        self.gx, self.gy = float(gx), float(gy)

    def init_equilibrium(self, rho=None, ux=None, uy=None):
        args = [_Arg(a, self.shape) for a in (rho, ux, uy)]
        dev = {a.device for a in args if a.ptr is not None}
        if len(dev) > 1:
            raise ValueError("mixing host and device arrays")
        self._check(self._lib.glbm_init_equilibrium(
            self._h, args[0].ptr, args[1].ptr, args[2].ptr, int(dev == {True})))

    def set_convergence(self, patience):
        """Converge only after `patience` consecutive passing checks."""
        self._check(self._lib.glbm_set_convergence(self._h, int(patience)))

    def step(self, n, tol=0.0, check_every=100):
        done, conv = C.c_longlong(), C.c_int()
        self._check(self._lib.glbm_step(self._h, int(n), float(tol),
                                        int(check_every), C.byref(done),
                                        C.byref(conv)))
        return done.value, bool(conv.value)

    def mean_velocity(self):
        out = (C.c_double * 2)()
        self._check(self._lib.glbm_mean_velocity(self._h, out))
        return np.array([out[0], out[1]])

    def permeability(self):
        k = C.c_double()
        self._check(self._lib.glbm_permeability(self._h, C.byref(k)))
        return k.value

    def velocity(self, ux=None, uy=None):
        """Eq. 34 velocity field of the last step -> (ux, uy); pass CUDA
        float64 tensors to keep the result on the device."""
        if ux is None:
            ux, uy = np.empty(self.shape), np.empty(self.shape)
        a, b = _Arg(ux, self.shape, True), _Arg(uy, self.shape, True)
        self._check(self._lib.glbm_get_velocity(self._h, a.ptr, b.ptr, int(a.device)))
        return ux, uy

    def distributions(self, out=None):
        """Absolute f_i in FP64, shape (9, ny, nx)."""
        shp = (9,) + self.shape
        if out is None:
            out = np.empty(shp)
        a = _Arg(out, shp, True)
        self._check(self._lib.glbm_get_distributions(self._h, a.ptr, int(a.device)))
        return out

    def save(self, path):
        """Checkpoint the whole solver state to a file (glbm_save)."""
        self._check(self._lib.glbm_save(self._h, os.fsencode(path)))

    def load(self, path):
        """Replace the solver state by a checkpoint of a solver of the same
        geometry, tau, storage and boundaries (glbm_load)."""
        self._check(self._lib.glbm_load(self._h, os.fsencode(path)))

    def counters(self):
        s, l = C.c_longlong(), C.c_longlong()
        self._check(self._lib.glbm_counters(self._h, C.byref(s), C.byref(l)))
        return s.value, l.value

    def guard_damage(self, poke=False):
        """Guard-zone bytes around the handle's device buffers that no longer
        hold their fill pattern (0 unless something wrote out of bounds);
        poke=True damages one byte first to show the count works."""
        d = C.c_longlong()
        self._check(self._lib.glbm_debug_guards(self._h, int(bool(poke)), C.byref(d)))
        return d.value


class Batch:
    """Many media of uneven size advanced together (a ``glbm_batch_t``).

    ``shapes`` is a list of (ny, nx) with nx a multiple of 4; ``storage`` is
    'f32' or 'bf16'.  Each medium matches a lone ``Solver`` bit for bit."""

    def __init__(self, shapes, tau=1.0, storage="f32", walls=True, stream=None):
        self._lib = load()
        self._h = _VP()
        self.shapes = [(int(ny), int(nx)) for ny, nx in shapes]
        self.tau = float(tau)
        n = len(self.shapes)
        nxs = (C.c_int * n)(*[nx for _, nx in self.shapes])
        nys = (C.c_int * n)(*[ny for ny, _ in self.shapes])
        st = STORAGE[storage] if isinstance(storage, str) else int(storage)
        sv = stream if (stream is None or isinstance(stream, int)) else stream.cuda_stream
        rc = self._lib.glbm_batch_create(n, nxs, nys, self.tau, st,
                                         WALLS_Y if walls else PERIODIC_Y,
                                         _VP(sv) if sv else None, C.byref(self._h))
        if rc != 0:
            raise GLBMError(rc, self._lib.glbm_batch_last_error(None).decode())

    def _check(self, rc):
        if rc != 0:
            raise GLBMError(rc, self._lib.glbm_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.glbm_batch_destroy(self._h)
            self._h = _VP()

    __del__ = close

    def __len__(self):
        return len(self.shapes)

    def set_medium(self, index, eps, K):
        shape = self.shapes[index]
        e, k = _Arg(eps, shape), _Arg(K, shape)
        if e.device != k.device:
            raise ValueError("eps and K must both be host or both device arrays")
        self._check(self._lib.glbm_batch_set_medium(self._h, int(index), e.ptr, k.ptr,
                                                    int(e.device)))

    def set_force(self, gx, gy=0.0):
        self._check(self._lib.glbm_batch_set_force(self._h, float(gx), float(gy)))

    def reset(self):
        self._check(self._lib.glbm_batch_reset(self._h))

    def set_schedule(self, threads, order):
        self._check(self._lib.glbm_batch_set_schedule(self._h, int(threads), int(order)))

    def set_convergence(self, patience):
        """A medium converges only after `patience` consecutive passing checks."""
        self._check(self._lib.glbm_batch_set_convergence(self._h, int(patience)))

    def set_persistent(self, on=True):
        """One cooperative launch per chunk with grid barriers between steps
        (True) or one launch per step from captured graphs (False)."""
        self._check(self._lib.glbm_batch_set_persistent(self._h, int(bool(on))))

    @property
    def persistent(self):
        v = C.c_int()
        self._check(self._lib.glbm_batch_get_persistent(self._h, C.byref(v)))
        return bool(v.value)

    def autotune(self, trial_steps=20):
        t, o = C.c_int(), C.c_int()
        self._check(self._lib.glbm_batch_autotune(self._h, int(trial_steps),
                                                  C.byref(t), C.byref(o)))
        return t.value, o.value

    def step(self, n, tol=0.0, check_every=100):
        done, left = C.c_longlong(), C.c_int()
        self._check(self._lib.glbm_batch_step(self._h, int(n), float(tol), int(check_every),
                                              C.byref(done), C.byref(left)))
        return done.value, left.value

    def guard_damage(self, poke=False):
        """As Solver.guard_damage, for the batch's device buffers."""
        d = C.c_longlong()
        self._check(self._lib.glbm_batch_debug_guards(self._h, int(bool(poke)), C.byref(d)))
        return d.value

    def results(self):
        """-> dict of per-medium arrays: kxx, mean_u (count x 2), steps, converged."""
        n = len(self.shapes)
        k = np.empty(n)
        u = np.empty((n, 2))
        st = np.empty(n, dtype=np.int64)
        cv = np.empty(n, dtype=np.int32)
        self._check(self._lib.glbm_batch_results(self._h, k.ctypes.data, u.ctypes.data,
                                                 st.ctypes.data, cv.ctypes.data))
        return {"kxx": k, "mean_u": u, "steps": st, "converged": cv.astype(bool)}

    def distributions(self, index):
        shape = (9,) + self.shapes[index]
        out = np.empty(shape)
        self._check(self._lib.glbm_batch_get_distributions(self._h, int(index),
                                                           out.ctypes.data, 0))
        return out

    def fields(self, index):
        """(rho, ux, uy) of medium `index` at its last step, FP64 (ny, nx) each."""
        shape = self.shapes[index]
        rho, ux, uy = np.empty(shape), np.empty(shape), np.empty(shape)
        self._check(self._lib.glbm_batch_get_fields(self._h, int(index), rho.ctypes.data,
                                                    ux.ctypes.data, uy.ctypes.data, 0))
        return rho, ux, uy

    def info(self):
        t, o, l, nn = C.c_int(), C.c_int(), C.c_longlong(), C.c_longlong()
        self._check(self._lib.glbm_batch_info(self._h, C.byref(t), C.byref(o), C.byref(l),
                                              C.byref(nn)))
        return {"threads": t.value, "order": o.value, "launches": l.value, "nodes": nn.value}


def em_gmm1d(x, phi, mu, var, max_iter=500, tol=1e-12):
    """EM fit of a 1-D Gaussian mixture on the GPU (Eqs. 20-24) -> (phi, mu,
    var, iterations, mean log-likelihood).  x: NumPy array or CUDA tensor."""
    lib = load()
    k = len(phi)
    p, u, v = ((C.c_double * k)(*map(float, a)) for a in (phi, mu, var))
    it, llv = C.c_int(), C.c_double()
    if _is_tensor(x) and x.is_cuda:
        import torch
        xs = x.to(torch.float64).contiguous()
        ptr, dev, n = xs.data_ptr(), 1, xs.numel()
    else:
        xs = np.ascontiguousarray(x, dtype=np.float64).ravel()
        ptr, dev, n = xs.ctypes.data, 0, xs.size
    rc = lib.glbm_em_gmm1d(ptr, n, k, p, u, v, int(max_iter), float(tol), C.byref(it),
                           C.byref(llv), dev, None)
    if rc != 0:
        raise GLBMError(rc, lib.glbm_last_error(None).decode())
    return np.array(p[:]), np.array(u[:]), np.array(v[:]), it.value, llv.value


def qsat_from_langmuir_volume(qsat_b, rho_b, eps, toc, rho_ch4, M_ch4=0.01604):
    """Eq. 38 (via the C ABI): Langmuir volume (m^3/kg) -> q_sat (mol/m^3)."""
    return load().glbm_qsat_from_langmuir_volume(float(qsat_b), float(rho_b), float(eps),
                                                 float(toc), float(rho_ch4), float(M_ch4))


def kapp_field(r, organic, eps, P, T, eta, tort, qsat, b, Ds, dx, M=0.01604):
    """Per-node DGM/GMS apparent permeability in lattice units (Eqs. 18-19):
    NumPy inputs of equal shape -> K_app / dx^2 as float64, same shape."""
    lib = load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    org = np.ascontiguousarray(organic, dtype=np.uint8)
    e = np.ascontiguousarray(eps, dtype=np.float64)
    if not (r.shape == org.shape == e.shape):
        raise ValueError("r, organic and eps must have one shape")
    K = np.empty_like(r)
    rc = lib.glbm_kapp_field(r.ctypes.data, org.ctypes.data, e.ctypes.data, r.size,
                             float(P), float(T), float(M), float(eta), float(tort),
                             float(qsat), float(b), float(Ds), float(dx),
                             K.ctypes.data, 0, None)
    if rc != 0:
        raise GLBMError(rc, lib.glbm_last_error(None).decode())
    return K
