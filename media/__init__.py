"""Seeded synthetic shale media for the generalized lattice Boltzmann model.

This module only *generates inputs*: per-node porosity eps(x) and apparent
permeability K(x) on a 2-D lattice, row-major ``[ny][nx]`` float64 arrays.
It holds none of the lattice Boltzmann arithmetic and imports neither the
CPU oracle nor the CUDA library, so both sides can draw identical media from
it.

The paper reconstructs its shale matrix from an Eagle Ford sample whose pore
data and reconstruction method it does not publish (Sec. 3.2, Sec. 3.3).  The
stand-in used here is a two-phase organic-matter (OM) / inorganic-matter (IOM)
map grown as clusters by thresholding a Gaussian random field:

* white noise from ``numpy.random.Generator(PCG64(seed))``;
* spectral filter ``exp(-|k|^2 l^2 / 4)`` on the periodic grid, i.e. a field
  with Gaussian covariance ``exp(-r^2 / (2 l^2))`` of correlation length l;
* the ``round(phi * N)`` largest field values become OM (ties broken by the
  linear node index, lowest first);
* per phase a constant porosity and a log-uniform permeability drawn
  independently per node (lattice units).

All randomness comes from the one seeded generator, in a fixed draw order
(noise field first, then the K uniforms), so a (shape, parameters, seed)
triple always yields the same arrays on one platform.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_random_field",
    "two_phase_map",
    "two_phase_medium",
    "uniform_medium",
    "layered_medium",
    "random_medium",
    "random_state",
    "shale_batch",
]


def gaussian_random_field(nx: int, ny: int, corr_len: float,
                          rng: np.random.Generator) -> np.ndarray:
    """Periodic Gaussian random field, shape (ny, nx), zero mean, unit variance."""
    noise = rng.standard_normal((ny, nx))
    kx = 2.0 * np.pi * np.fft.rfftfreq(nx)
    ky = 2.0 * np.pi * np.fft.fftfreq(ny)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    spec = np.fft.rfft2(noise) * np.exp(-k2 * (corr_len ** 2) / 4.0)
    field = np.fft.irfft2(spec, s=(ny, nx))
    field -= field.mean()
    sd = field.std()
    if sd > 0:
        field /= sd
    return field


def two_phase_map(nx: int, ny: int, om_fraction: float, corr_len: float,
                  rng: np.random.Generator) -> np.ndarray:
    """Boolean OM mask (True = organic matter) with exactly round(phi*N) OM nodes."""
    if not 0.0 <= om_fraction <= 1.0:
        raise ValueError("om_fraction must lie in [0, 1]")
    field = gaussian_random_field(nx, ny, corr_len, rng).ravel()
    n = field.size
    n_om = int(round(om_fraction * n))
    mask = np.zeros(n, dtype=bool)
    if n_om > 0:
        # the n_om-th largest value, then every larger value plus the lowest
        # linear indices among values equal to it (same set as a stable sort)
        thr = np.partition(field, n - n_om)[n - n_om]
        mask = field > thr
        ties = np.flatnonzero(field == thr)
        mask[ties[:n_om - int(mask.sum())]] = True
    return mask.reshape(ny, nx)


def _log_uniform(u: np.ndarray, lo: float, hi: float) -> np.ndarray:
    a, b = np.log10(lo), np.log10(hi)
    return 10.0 ** (a + u * (b - a))


def two_phase_medium(nx: int, ny: int, *, om_fraction: float = 0.2,
                     corr_len: float = 8.0, seed: int = 0,
                     eps_iom: float = 0.10, eps_om: float = 0.15,
                     k_iom: tuple[float, float] = (1e-4, 1e-3),
                     k_om: tuple[float, float] = (5e-4, 5e-3)):
    """Two-phase OM/IOM medium: returns (eps, K, om_mask), each shaped (ny, nx).

    Defaults are the 128x128 / 4096x4096 workloads: OM fraction 0.2 grown
    with correlation length 8 nodes, eps 0.10 (IOM) / 0.15 (OM), K
    log-uniform in [1e-4, 1e-3] (IOM) and [5e-4, 5e-3] (OM), lattice units.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    om = two_phase_map(nx, ny, om_fraction, corr_len, rng)
    u = rng.random((ny, nx))
    eps = np.where(om, eps_om, eps_iom).astype(np.float64)
    K = np.where(om, _log_uniform(u, *k_om), _log_uniform(u, *k_iom))
    return np.ascontiguousarray(eps), np.ascontiguousarray(K), om


def uniform_medium(nx: int, ny: int, eps: float, K: float):
    """Homogeneous medium (K may be +inf for a clear fluid)."""
    return (np.full((ny, nx), float(eps)), np.full((ny, nx), float(K)))


def layered_medium(nx: int, ny: int, layers, axis: str):
    """Stacked homogeneous layers.

    ``layers`` is a sequence of (thickness, eps, K).  ``axis='x'`` stacks them
    along x (layers perpendicular to a flow along x, i.e. in series);
    ``axis='y'`` stacks them along y (layers parallel to the flow).  The
    thicknesses must add up to nx or ny respectively.
    """
    eps = np.empty((ny, nx))
    K = np.empty((ny, nx))
    pos = 0
    for t, e, k in layers:
        if axis == "x":
            eps[:, pos:pos + t] = e
            K[:, pos:pos + t] = k
        elif axis == "y":
            eps[pos:pos + t, :] = e
            K[pos:pos + t, :] = k
        else:
            raise ValueError("axis must be 'x' or 'y'")
        pos += t
    if pos != (nx if axis == "x" else ny):
        raise ValueError("layer thicknesses do not cover the lattice")
    return eps, K


def random_medium(nx: int, ny: int, seed: int, *, eps_range=(0.05, 1.0),
                  k_range=(1e-3, 1e1)):
    """I.i.d. per-node eps (uniform) and K (log-uniform): a stress input for
    step-by-step comparisons, with large velocities so every term matters."""
    rng = np.random.Generator(np.random.PCG64(seed))
    eps = rng.uniform(eps_range[0], eps_range[1], size=(ny, nx))
    K = _log_uniform(rng.random((ny, nx)), *k_range)
    return eps, K


def random_state(nx: int, ny: int, seed: int, *, amp: float = 1e-3,
                 u_amp: float = 0.02):
    """Seeded smooth-ish initial (rho, ux, uy) fields for warm-start tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = 1.0 + amp * rng.standard_normal((ny, nx))
    ux = u_amp * rng.standard_normal((ny, nx))
    uy = u_amp * rng.standard_normal((ny, nx))
    return rho, ux, uy


def shale_batch(count: int = 512, *, seed: int = 0, sides=tuple(range(64, 1025, 64)),
                om_fraction: float = 0.2, corr_len: float = 8.0,
                r_median=(20e-9, 5e-9), sigma_ln: float = 0.5,
                eps_phase=(0.02, 0.04), pressure=(0.5e6, 30e6),
                langmuir_pressure=(2e6, 10e6), langmuir_volume=(0.002, 0.01)):
    """Inputs of a batched sweep over shale media (one dict per medium).

    Per medium: a square side drawn uniformly from ``sides``; an OM/IOM map
    grown as in ``two_phase_map``; per-node pore radius lognormal around the
    phase median (IOM first, OM second) with log-standard deviation
    ``sigma_ln``; per-phase porosity; a pressure uniform in ``pressure`` (Pa);
    a Langmuir pressure P_L uniform in ``langmuir_pressure`` (b = 1/P_L) and a
    Langmuir volume V_L uniform in ``langmuir_volume`` (m^3/kg).  Everything
    comes from one PCG64(seed) stream in a fixed order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        n = int(rng.choice(sides))
        om = two_phase_map(n, n, om_fraction, corr_len, rng)
        z = rng.standard_normal((n, n))
        med = np.where(om, r_median[1], r_median[0])
        r = med * np.exp(sigma_ln * z)
        eps = np.where(om, eps_phase[1], eps_phase[0]).astype(np.float64)
        out.append({
            "n": n, "organic": om, "r": r, "eps": eps,
            "P": float(rng.uniform(*pressure)),
            "P_L": float(rng.uniform(*langmuir_pressure)),
            "V_L": float(rng.uniform(*langmuir_volume)),
            "toc": float(om.mean()),
        })
    return out
