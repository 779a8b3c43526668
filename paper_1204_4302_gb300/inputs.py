"""Seeded synthetic magnetization states, shared by the tests, the benchmark
and the oracle checks.

This module only draws inputs. It holds none of the stray-field arithmetic and
imports nothing from the library or from the oracle. All arrays are float64
numpy arrays of shape (3, nz, ny, nx) with x fastest (SoA, C order).

States of the paper's experiments (Sec. 5):
  * homogeneous cube / film (Sec. 5.1, 5.3),
  * flower state in a cube (Sec. 5.2, Eq. "flower_mag", a = c = 1, b = 2),
  * vortex state (Sec. 5.2, Eq. "config1", Feldtkeller profile, r_c = 0.14),
  * homogeneous sphere on a staircase grid (Sec. 5.4: cells whose centre lies
    inside the sphere carry M = (0, 0, Mz), the others zero).
Cell centres are sampled with the body centred at the origin.
"""
from __future__ import annotations

import numpy as np


def cell_centres(n, extent):
    """Centres of an nx x ny x nz grid spanning a box of the given extent
    centred at the origin; returns (X, Y, Z) each of shape (nz, ny, nx)."""
    nx, ny, nz = (int(v) for v in n)
    Lx, Ly, Lz = (float(v) for v in extent)
    x = (np.arange(nx) + 0.5) * (Lx / nx) - 0.5 * Lx
    y = (np.arange(ny) + 0.5) * (Ly / ny) - 0.5 * Ly
    z = (np.arange(nz) + 0.5) * (Lz / nz) - 0.5 * Lz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def normalise(m: np.ndarray) -> np.ndarray:
    nrm = np.sqrt(np.sum(m * m, axis=0, keepdims=True))
    nrm[nrm == 0] = 1.0
    return m / nrm


def uniform(n, direction=(1.0, 0.0, 0.0)) -> np.ndarray:
    nx, ny, nz = (int(v) for v in n)
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    m = np.empty((3, nz, ny, nx))
    for c in range(3):
        m[c] = d[c]
    return m


def random_unit(n, seed: int) -> np.ndarray:
    """Independent unit vectors per cell: a standard normal 3-vector, normalised."""
    nx, ny, nz = (int(v) for v in n)
    rng = np.random.default_rng(seed)
    m = rng.standard_normal((3, nz, ny, nx))
    return normalise(m)


def flower(n, extent=(1.0, 1.0, 1.0), a=1.0, b=2.0, c=1.0) -> np.ndarray:
    """Normalised m ~ (x z / a, y z / c + y^3 z^3 / b^3, 1) (paper Sec. 5.2)."""
    X, Y, Z = cell_centres(n, extent)
    m = np.stack([X * Z / a, Y * Z / c + (Y ** 3) * (Z ** 3) / b ** 3, np.ones_like(X)])
    return normalise(m)


def vortex(n, extent=(1.0, 1.0, 1.0), rc=0.14) -> np.ndarray:
    """Feldtkeller vortex about the z axis (paper Sec. 5.2): in-plane curl with
    weight sqrt(1 - exp(-4 r^2/rc^2)), out-of-plane core exp(-2 r^2/rc^2).
    At r = 0 the state is (0, 0, 1)."""
    X, Y, _ = cell_centres(n, extent)
    r2 = X * X + Y * Y
    r = np.sqrt(r2)
    safe = np.where(r > 0, r, 1.0)
    w = np.sqrt(1.0 - np.exp(-4.0 * r2 / rc ** 2))
    mx = np.where(r > 0, -Y / safe * w, 0.0)
    my = np.where(r > 0, X / safe * w, 0.0)
    mz = np.exp(-2.0 * r2 / rc ** 2)
    return np.stack([mx, my, mz])


def vortex_noise(n, extent, rc, noise: float, seed: int) -> np.ndarray:
    """Vortex plus independent Gaussian noise of the given standard deviation per
    component, renormalised."""
    m = vortex(n, extent, rc)
    rng = np.random.default_rng(seed)
    m = m + noise * rng.standard_normal(m.shape)
    return normalise(m)


def sphere_mask(n, radius_cells: float) -> np.ndarray:
    """1 for cells whose centre lies strictly inside a sphere of the given radius
    (in cells) centred in the grid, else 0. Shape (nz, ny, nx)."""
    nx, ny, nz = (int(v) for v in n)
    X, Y, Z = cell_centres(n, (nx, ny, nz))
    return ((X * X + Y * Y + Z * Z) < radius_cells ** 2).astype(np.float64)


def smooth_random(n, corr_cells: float, seed: int) -> np.ndarray:
    """Gaussian-filtered white noise per component (periodic, separable filter of
    standard deviation corr_cells), normalised per cell."""
    nx, ny, nz = (int(v) for v in n)
    rng = np.random.default_rng(seed)
    m = rng.standard_normal((3, nz, ny, nx))
    for axis, L in ((3, nx), (2, ny), (1, nz)):
        k = np.fft.fftfreq(L)
        g = np.exp(-2.0 * (np.pi * k * corr_cells) ** 2)
        shape = [1, 1, 1, 1]
        shape[axis] = L
        m = np.real(np.fft.ifft(np.fft.fft(m, axis=axis) * g.reshape(shape), axis=axis))
    return normalise(m)


def batch_sizes(count: int, lo=(32, 32, 8), hi=(128, 128, 32), seed: int = 4):
    """Per-state grid sizes (nx, ny, nz), each axis uniform on [lo, hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        out.append(tuple(int(rng.integers(lo[a], hi[a] + 1)) for a in range(3)))
    return out
