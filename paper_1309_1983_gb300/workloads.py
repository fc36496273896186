"""Seeded synthetic inputs for the D3Q19 lattice Boltzmann workloads.

This module is shared by the CUDA path's tests and benchmark and by the FP64
oracle's tests. It holds no arithmetic of the lattice Boltzmann method (no
velocity set, weights, equilibrium or collision): only the initial and target
velocity fields, force fields, noise and batch geometries that the workloads
are defined by. Every array is float64 and laid out as planes
``(3, nz, ny, nx)`` (vector fields) or ``(nz, ny, nx)`` (scalars).

The workloads are the synthetic ones the paper benchmarks on (a lid-driven
cubic cavity, Sec. 5 and Sec. 6) plus periodic shear waves, random Fourier
velocity fields and batches of uneven cavities.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def shear_wave(nx: int, ny: int, nz: int, amp: float = 0.01) -> np.ndarray:
    """u_x(z) = amp * sin(2 pi z / nz), u_y = u_z = 0."""
    u = np.zeros((3, nz, ny, nx), dtype=np.float64)
    z = np.arange(nz, dtype=np.float64)
    u[0] = (amp * np.sin(2.0 * np.pi * z / nz))[:, None, None]
    return u


def fourier_modes(nx: int, ny: int, nz: int, seed: int, kmax: float = 4.0,
                  amp: float = 0.02) -> np.ndarray:
    """A random periodic velocity field: the sum, over every integer wave
    vector k with 0 < |k| <= kmax, of a_k cos(2 pi k.x / n) + b_k sin(...),
    with a_k, b_k independent standard-normal 3-vectors drawn from
    ``numpy.random.default_rng(seed)`` in a fixed k order, then scaled so
    that max_x |u(x)| = amp. No divergence projection is applied."""
    rng = np.random.default_rng(seed)
    r = int(np.floor(kmax))
    ks = [(kx, ky, kz)
          for kz in range(-r, r + 1) for ky in range(-r, r + 1) for kx in range(-r, r + 1)
          if 0 < kx * kx + ky * ky + kz * kz <= kmax * kmax]
    coef = np.zeros((3, nz, ny, nx), dtype=np.complex128)
    for (kx, ky, kz) in ks:
        a = rng.standard_normal(3)
        b = rng.standard_normal(3)
        # a cos(t) + b sin(t) = Re[(a - i b) exp(i t)]
        coef[:, kz % nz, ky % ny, kx % nx] += a - 1j * b
    u = np.empty((3, nz, ny, nx), dtype=np.float64)
    for c in range(3):
        u[c] = np.real(np.fft.ifftn(coef[c])) * (nx * ny * nz)
    speed = np.sqrt((u * u).sum(axis=0)).max()
    if speed > 0:
        u *= amp / speed
    return u


def noise(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Uniform noise in [-scale, scale) of the given shape."""
    rng = np.random.default_rng(seed)
    return scale * (2.0 * rng.random(shape) - 1.0)


def uniform_force(nx: int, ny: int, nz: int, F=(0.0, 0.0, 0.0)) -> np.ndarray:
    f = np.zeros((3, nz, ny, nx), dtype=np.float64)
    for a in range(3):
        f[a] = F[a]
    return f


@dataclass
class BatchGeometry:
    dims: np.ndarray    # (ndom, 3) int: nx, ny, nz per domain
    tau: np.ndarray     # (ndom,)
    lid_u: np.ndarray   # (ndom,) lid speed along +x


def batch_geometry(ndom: int = 64, seed: int = 3, edge=(16, 96), tau=(0.55, 1.0),
                   lid=(0.02, 0.08)) -> BatchGeometry:
    """Uneven cavities: edge lengths uniform integers in [edge[0], edge[1]]
    per axis, tau uniform in [tau[0], tau[1]), lid speed uniform in
    [lid[0], lid[1]), all from ``numpy.random.default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    dims = rng.integers(edge[0], edge[1] + 1, size=(ndom, 3))
    t = rng.uniform(tau[0], tau[1], size=ndom)
    l = rng.uniform(lid[0], lid[1], size=ndom)
    return BatchGeometry(dims=dims.astype(np.int64), tau=t, lid_u=l)


def separable_modes(nx: int, ny: int, nz: int, seed: int, modes: int = 4,
                    amp: float = 0.02, dtype=np.float32) -> np.ndarray:
    """A cheap random periodic velocity field for large lattices: for each
    component, the sum of ``modes`` products sin(2 pi (k_x x/nx + a)) *
    sin(2 pi (k_y y/ny + b)) * sin(2 pi (k_z z/nz + c)) with integer
    k in [1, 4] and phases from ``numpy.random.default_rng(seed)``, each term
    scaled by amp / modes (so |u_a| <= amp)."""
    rng = np.random.default_rng(seed)
    u = np.zeros((3, nz, ny, nx), dtype=dtype)
    x = np.arange(nx) / nx
    y = np.arange(ny) / ny
    z = np.arange(nz) / nz
    for c in range(3):
        for _ in range(modes):
            k = rng.integers(1, 5, size=3)
            ph = rng.random(3)
            sx = np.sin(2 * np.pi * (k[0] * x + ph[0])).astype(dtype)
            sy = np.sin(2 * np.pi * (k[1] * y + ph[1])).astype(dtype)
            sz = np.sin(2 * np.pi * (k[2] * z + ph[2])).astype(dtype)
            u[c] += (amp / modes) * sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    return u
