"""CPU oracle of the generalized lattice Boltzmann model (GLBM), Sec. 2.3.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only ``tests/``, the smoke check and
the benchmark's CPU-baseline leg may import this package.  It never imports
the CUDA library and the CUDA library never imports it.

The arithmetic lives in ``glbm_oracle.c`` (plain FP64 C, one node at a time,
absolute distributions); this module compiles it with gcc and wraps it with
ctypes.  Two builds come from the one source: a single-thread build for
parity and an OpenMP build (rows in parallel) for timing; both give the same
bits.

Parity status per function (pins in ``tests/test_oracle_*.py``):

* ``equilibrium``      - pinned: moments 0, 1, 2 against the ε-equilibrium
                         moment definitions.
* ``forcing``          - pinned: moments 0, 1, 2 against the Guo-Zhao forcing
                         moments.
* ``velocity``         - pinned: satisfies Eq. 33 with F from Eq. 27.
* ``run``              - pinned: Darcy and Forchheimer fixed points,
                         Poiseuille (exact at tau = 1/2 + sqrt(3)/4),
                         Brinkman channel (2nd-order convergence), series
                         layers (exact momentum balance), Taylor-Green decay
                         (viscosity), mass conservation, D2Q9 BGK+Guo
                         textbook reduction (eps = 1, K = inf).
* two-phase random media (the benchmark workload) - no closed form for the
  fields; pinned by the exact domain momentum balance (sum of rho F = 0 at
  steady state, F from Eq. 27, with and without Forchheimer drag) besides
  the invariants above.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glbm_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "dgm_gms.c"), os.path.join(_HERE, "em_gmm.c")]
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[bool, C.CDLL] = {}

_D = C.c_double
_PD = C.POINTER(C.c_double)


def _lib_path(omp: bool) -> str:
    return os.path.join(_BUILD, "liboracle_omp.so" if omp else "liboracle.so")


def build(force: bool = False) -> None:
    """Compile both oracle builds with gcc (FP contraction off, so x86 and
    Arm hosts produce the same bits)."""
    os.makedirs(_BUILD, exist_ok=True)
    for omp in (False, True):
        out = _lib_path(omp)
        srcs = [p for p in _SRCS if os.path.exists(p)]
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= max(os.path.getmtime(p) for p in srcs)):
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", *srcs, "-o", tmp, "-lm"]
        if omp:
            cmd.insert(1, "-fopenmp")
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


def _lib(omp: bool = False) -> C.CDLL:
    with _LOCK:
        if omp not in _LIBS:
            if not os.path.exists(_lib_path(omp)):
                build()
            lib = C.CDLL(_lib_path(omp))
            lib.orc_run.restype = C.c_int
            lib.orc_run.argtypes = [
                C.c_int, C.c_int, _D, C.c_int, C.c_int, _PD, _PD, _D, _D, _D,
                _PD, C.c_longlong, _D, C.c_int, _PD, _PD, _PD, _PD, _PD,
                C.POINTER(C.c_longlong), C.POINTER(C.c_int)]
            lib.orc_equilibrium.argtypes = [_D, _D, _D, _D, _PD]
            lib.orc_forcing.argtypes = [_D, _D, _D, _D, _D, _D, _D, C.c_int, _PD]
            lib.orc_velocity.argtypes = [_D, _D, _D, _D, _D, _D, _D, _D, _D,
                                         _PD, _PD]
            lib.orc_body_force.argtypes = [_D, _D, _D, _D, _D, _D, _D, _D,
                                           _PD, _PD]
            lib.orc_c0_c1.argtypes = [_D, _D, _D, _D, _PD, _PD]
            lib.orc_feps.restype = _D
            lib.orc_feps.argtypes = [_D, _D]
            lib.orc_init_equilibrium.argtypes = [C.c_int, C.c_int, _PD, _PD,
                                                 _PD, _PD, _PD]
            lib.orc_permeability.restype = _D
            lib.orc_permeability.argtypes = [_D, _D, _D]
            lib.orc_threads.restype = C.c_int
            lib.orc_threads.argtypes = [C.c_int]
            lib.orc_dgm_kc_k0.argtypes = [_D, _D, _D, _PD, _PD]
            lib.orc_knudsen_diffusivity.restype = _D
            lib.orc_knudsen_diffusivity.argtypes = [_D, _D, _D]
            lib.orc_kapp.restype = _D
            lib.orc_kapp.argtypes = [_D] * 7 + [C.c_int] + [_D] * 3
            lib.orc_qsat_from_langmuir_volume.restype = _D
            lib.orc_qsat_from_langmuir_volume.argtypes = [_D] * 6
            lib.orc_em_gmm1d.restype = C.c_int
            lib.orc_em_gmm1d.argtypes = [_PD, C.c_long, C.c_int, _PD, _PD, _PD, C.c_int, _D, _PD]
            lib.orc_kapp_field.argtypes = [_PD, C.POINTER(C.c_ubyte), _PD, C.c_long] + [_D] * 9 + [_PD]
            _LIBS[omp] = lib
        return _LIBS[omp]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_PD)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# D2Q9 weights in the oracle's direction order, for callers that convert
# between absolute distributions and deviations.
WEIGHTS = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def equilibrium(rho, ux, uy, eps):
    """Eq. 30 at one node -> array of 9."""
    out = np.zeros(9)
    _lib().orc_equilibrium(rho, ux, uy, eps, _ptr(out))
    return out


def forcing(rho, ux, uy, Fx, Fy, eps, tau, literal=False):
    """Eq. 31 at one node -> array of 9 (``literal`` keeps the printed
    -3(u.F) last term instead of -(3/eps)(u.F))."""
    out = np.zeros(9)
    _lib().orc_forcing(rho, ux, uy, Fx, Fy, eps, tau, int(literal), _ptr(out))
    return out


def velocity(rho, mx, my, eps, K, feps, nu, gx, gy):
    """Eqs. 35, 36, 37, 34 at one node -> (ux, uy)."""
    ux, uy = _D(), _D()
    _lib().orc_velocity(rho, mx, my, eps, K, feps, nu, gx, gy,
                        C.byref(ux), C.byref(uy))
    return ux.value, uy.value


def body_force(ux, uy, eps, K, feps, nu, gx, gy):
    """Eq. 27 at one node -> (Fx, Fy)."""
    Fx, Fy = _D(), _D()
    _lib().orc_body_force(ux, uy, eps, K, feps, nu, gx, gy,
                          C.byref(Fx), C.byref(Fy))
    return Fx.value, Fy.value


def c0_c1(eps, K, feps, nu):
    a, b = _D(), _D()
    _lib().orc_c0_c1(eps, K, feps, nu, C.byref(a), C.byref(b))
    return a.value, b.value


def feps(mode, eps):
    return _lib().orc_feps(mode, eps)


def permeability(tau, mean_ux, gx):
    """Darcy upscaling K_app = nu <u_x> / G_x (lattice units)."""
    return _lib().orc_permeability(tau, mean_ux, gx)


def init_equilibrium(eps, rho=None, ux=None, uy=None):
    """Distributions f = f_eq(rho, u; eps) per node, shape (9, ny, nx)."""
    eps = _f64(eps)
    ny, nx = eps.shape
    f = np.zeros((9, ny, nx))
    _lib().orc_init_equilibrium(nx, ny, _ptr(eps), _ptr(_f64(rho)),
                                _ptr(_f64(ux)), _ptr(_f64(uy)), _ptr(f))
    return f


# -- DGM/GMS apparent permeability (Sec. 2.1) --------------------------------

METHANE_M = 0.01604  # kg/mol


def dgm_kc_k0(r, eps, tort):
    """Eq. 4 -> (K_c, K0) for pore radius r."""
    a, b = _D(), _D()
    _lib().orc_dgm_kc_k0(r, eps, tort, C.byref(a), C.byref(b))
    return a.value, b.value


def knudsen_diffusivity(Kc, T, M=METHANE_M):
    """Eq. 3."""
    return _lib().orc_knudsen_diffusivity(Kc, T, M)


def kapp(r, P, T, eta, eps, tort, organic, qsat=0.0, b=0.0, Ds=0.0, M=METHANE_M):
    """Eq. 18 (organic=False) or Eq. 19 (organic=True), SI units, m^2."""
    return _lib().orc_kapp(r, P, T, M, eta, eps, tort, int(bool(organic)),
                           qsat, b, Ds)


def qsat_from_langmuir_volume(qsat_b, rho_b, eps, toc, rho_ch4, M_ch4=METHANE_M):
    """Eq. 38: Langmuir volume (m^3/kg) -> q_sat (mol/m^3 of kerogen)."""
    return _lib().orc_qsat_from_langmuir_volume(qsat_b, rho_b, eps, toc,
                                                rho_ch4, M_ch4)


def kapp_field(r, organic, eps, P, T, eta, tort, qsat, b, Ds, dx, M=METHANE_M):
    """Per-node K_app / dx^2 (lattice units) for arrays r, organic, eps."""
    r = _f64(r)
    org = np.ascontiguousarray(organic, dtype=np.uint8)
    e = _f64(eps)
    K = np.empty_like(r)
    _lib().orc_kapp_field(_ptr(r), org.ctypes.data_as(C.POINTER(C.c_ubyte)),
                          _ptr(e), r.size, P, T, M, eta, tort, qsat, b, Ds, dx,
                          _ptr(K))
    return K


# -- EM for a 1-D Gaussian mixture (Sec. 2.2) ----------------------------------

def em_gmm1d(x, phi, mu, var, max_iter=500, tol=0.0):
    """Eqs. 20-24 from the initial guess (phi, mu, var) -> (phi, mu, var,
    iterations, mean log-likelihood of the last E-step)."""
    x = _f64(x).ravel()
    phi, mu, var = (np.array(a, dtype=np.float64) for a in (phi, mu, var))
    ll = _D()
    it = _lib().orc_em_gmm1d(_ptr(x), x.size, phi.size, _ptr(phi), _ptr(mu), _ptr(var),
                             int(max_iter), float(tol), C.byref(ll))
    if it < 0:
        raise ValueError("orc_em_gmm1d: bad arguments")
    return phi, mu, var, it, ll.value


class Oracle:
    """Stateful FP64 GLBM run on the CPU, mirroring the library's life cycle
    (set_medium -> set_force -> step* -> mean_velocity/permeability)."""

    def __init__(self, nx, ny, tau=1.0, periodic_y=False, literal=False,
                 threads: int | None = None):
        if nx < 2 or ny < 2 or not tau > 0.5:
            raise ValueError("need nx, ny >= 2 and tau > 1/2")
        self.nx, self.ny, self.tau = nx, ny, float(tau)
        self.periodic_y, self.literal = bool(periodic_y), bool(literal)
        self.omp = threads is not None
        if self.omp:
            _lib(True).orc_threads(int(threads))
        self.gx = self.gy = 0.0
        self.feps_mode = 0.0
        self.eps = self.K = self.f = None
        self.ux = self.uy = self.rho = None
        self.mean_u = np.zeros(2)
        self.conv_state = np.zeros(2)
        self.steps = 0

    @property
    def nu(self):
        return (self.tau - 0.5) / 3.0

    def set_medium(self, eps, K, feps_mode=0.0):
        eps, K = _f64(eps), _f64(K)
        if eps.shape != (self.ny, self.nx) or K.shape != eps.shape:
            raise ValueError("eps and K must be shaped (ny, nx)")
        self.eps, self.K = eps, K
        self.feps_mode = float(feps_mode)
        self.init_equilibrium()

    def set_force(self, gx, gy=0.0):
        self.gx, self.gy = float(gx), float(gy)
        self.conv_state[:] = 0.0

    def init_equilibrium(self, rho=None, ux=None, uy=None):
        self.f = init_equilibrium(self.eps, rho, ux, uy)
        self.steps = 0
        self.conv_state[:] = 0.0
        self.ux = self.uy = self.rho = None

    def step(self, n, tol=0.0, check_every=100):
        self.ux = np.zeros((self.ny, self.nx))
        self.uy = np.zeros((self.ny, self.nx))
        self.rho = np.zeros((self.ny, self.nx))
        done, conv = C.c_longlong(), C.c_int()
        rc = _lib(self.omp).orc_run(
            self.nx, self.ny, self.tau, int(self.periodic_y),
            int(self.literal), _ptr(self.eps), _ptr(self.K), self.feps_mode,
            self.gx, self.gy, _ptr(self.f), int(n), float(tol),
            int(check_every), _ptr(self.ux), _ptr(self.uy), _ptr(self.rho),
            _ptr(self.mean_u), _ptr(self.conv_state), C.byref(done),
            C.byref(conv))
        if rc == -4:
            raise FloatingPointError("non-finite mean velocity")
        if rc != 0:
            raise RuntimeError(f"orc_run failed with {rc}")
        self.steps += done.value
        return done.value, bool(conv.value)

    def permeability(self):
        return permeability(self.tau, self.mean_u[0], self.gx)

    def deviations(self):
        """Current state as deviations g_i = f_i - w_i (rho0 = 1)."""
        return self.f - WEIGHTS[:, None, None]
