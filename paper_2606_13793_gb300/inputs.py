"""Seeded synthetic densities shaped like the paper's test problems.

This module holds input generators only -- no step of the FMM -- so that the
oracle-side tests and the CUDA-side tests and benchmark can draw identical
inputs from it.  Every generator is deterministic in its seed.

The paper's tests (Sec. 3, App. B) use a point charge, two uniform spheres and
an NFW halo deposited on 256^3 grids; the densities below stand in for those
and for the benchmark workloads (none of the paper's particle data exists
here):

* ``gaussian_blobs``  -- a few Gaussian blobs (smooth, compact mass).
* ``lognormal``       -- exp of a Gaussian random field with P(k) ~ k^slope,
                         outer margin zeroed so the mass is compact (a
                         cosmological-looking clustered field).
* ``plummer``         -- a centred Plummer sphere plus 1% uniform noise.
* ``point_mass``, ``uniform_spheres`` -- the paper's two closed-form set-ups.
"""
from __future__ import annotations

import numpy as np

__all__ = ["gaussian_blobs", "lognormal", "plummer", "point_mass", "uniform_spheres", "batch_sizes"]


def _centres(shape):
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    return x, y, z


def _shape3(n):
    if np.isscalar(n):
        return (int(n), int(n), int(n))
    return tuple(int(v) for v in n)


def gaussian_blobs(n, seed: int = 2606, count: int = 3, sigma=(2.0, 5.0), mass=(0.5, 2.0), dtype=np.float64):
    """rho = sum_k M_k (2 pi s_k^2)^-3/2 exp(-|x-c_k|^2 / 2 s_k^2) at cell centres.

    Centres uniform in the box, s_k ~ U[sigma], M_k ~ U[mass] (cell units).
    Returned as [nz][ny][nx].
    """
    shape = _shape3(n)
    rng = np.random.default_rng(seed)
    x, y, z = _centres(shape)
    rho = np.zeros(x.shape, dtype=np.float64)
    for _ in range(count):
        c = rng.uniform(0.0, 1.0, 3) * np.array(shape, dtype=np.float64)
        s = rng.uniform(*sigma)
        m = rng.uniform(*mass)
        r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
        rho += m * (2.0 * np.pi * s * s) ** -1.5 * np.exp(-0.5 * r2 / (s * s))
    return rho.astype(dtype)


def lognormal(n, seed: int = 2606, slope: float = -2.5, pad_frac: float = 0.1, dtype=np.float32):
    """Lognormal transform of a seeded Gaussian random field.

    delta has power spectrum P(k) ~ k^slope (k = 0 mode removed), built by
    FFT of seeded white noise and normalised to unit variance; rho =
    exp(delta - 1/2).  Every cell with min(i, n-1-i) < floor(pad_frac * n)
    on any axis is zeroed, so the mass is compact (isolated boundaries).
    """
    import scipy.fft as sfft

    shape = _shape3(n)
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((nz, ny, nx), dtype=np.float32)
    wk = sfft.rfftn(white, workers=-1)
    del white
    kz = np.fft.fftfreq(nz).astype(np.float32)[:, None, None]
    ky = np.fft.fftfreq(ny).astype(np.float32)[None, :, None]
    kx = np.fft.rfftfreq(nx).astype(np.float32)[None, None, :]
    k2 = kz * kz + ky * ky + kx * kx
    k2[0, 0, 0] = 1.0
    amp = k2 ** np.float32(slope / 4.0)  # sqrt(P) = k^(slope/2)
    amp[0, 0, 0] = 0.0
    wk *= amp
    del amp, k2
    delta = sfft.irfftn(wk, s=(nz, ny, nx), workers=-1).astype(np.float32)
    del wk
    delta -= delta.mean(dtype=np.float64)
    delta /= np.float32(delta.std(dtype=np.float64))
    rho = np.exp(delta - np.float32(0.5), dtype=np.float32)
    del delta
    for axis, m in zip((2, 1, 0), (nx, ny, nz)):
        pad = int(np.floor(pad_frac * m))
        if pad <= 0:
            continue
        sl = [slice(None)] * 3
        sl[axis] = slice(0, pad)
        rho[tuple(sl)] = 0.0
        sl[axis] = slice(m - pad, m)
        rho[tuple(sl)] = 0.0
    return rho.astype(dtype, copy=False)


def plummer(n, seed: int = 2606, a_range=(4.0, 20.0), total_mass: float = 1.0, noise: float = 0.01,
            dtype=np.float32):
    """Centred Plummer sphere rho = 3M/(4 pi a^3) (1 + r^2/a^2)^-5/2, a ~ U[a_range],
    plus uniform noise U[0, noise * rho_0) with rho_0 the central density."""
    shape = _shape3(n)
    rng = np.random.default_rng(seed)
    a = rng.uniform(*a_range)
    x, y, z = _centres(shape)
    c = np.array(shape, dtype=np.float64) / 2.0
    r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
    rho0 = 3.0 * total_mass / (4.0 * np.pi * a ** 3)
    rho = rho0 * (1.0 + r2 / (a * a)) ** -2.5
    rho += rng.uniform(0.0, noise * rho0, size=rho.shape)
    return rho.astype(dtype)


def point_mass(n, cell, mass: float = 1.0, dtype=np.float64):
    """All mass in one cell (the paper's single-charge test, without CIC)."""
    shape = _shape3(n)
    rho = np.zeros((shape[2], shape[1], shape[0]), dtype=dtype)
    i, j, k = cell
    rho[k, j, i] = mass
    return rho


def uniform_spheres(n, spheres, dtype=np.float64):
    """Cells whose centre lies inside a sphere get that sphere's density.

    ``spheres`` = [((cx, cy, cz), radius, density), ...] in cell units (the
    paper's two-sphere test uses two of these, Sec. 3)."""
    shape = _shape3(n)
    x, y, z = _centres(shape)
    rho = np.zeros(x.shape, dtype=np.float64)
    for (cx, cy, cz), r, d in spheres:
        inside = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= r * r
        rho[inside] += d
    return rho.astype(dtype)


def batch_sizes(count: int = 64, seed: int = 2606, choices=(64, 96, 128, 192)):
    """Seeded draw of per-field grid sizes for the uneven batch workload."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.choice(np.array(choices), size=count)]
