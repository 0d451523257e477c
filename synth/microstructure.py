"""Periodic two-phase microstructures (phase 0 = matrix, phase 1 = inclusion), seeded.

Voxel (x, y[, z]) has its centre at the integer coordinates; it belongs to an inclusion when
that centre lies inside the disc/sphere (periodic distance). Random composites use random
sequential addition of non-overlapping inclusions with a minimum periodic gap of one voxel,
repeated until the voxelised volume fraction reaches the target (or the attempt budget runs out).
Arrays are C-ordered with x fastest: shape (Ny, Nx) in 2D, (Nz, Ny, Nx) in 3D, dtype uint8.
"""

from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def centred_disc(n: int, vf: float) -> np.ndarray:
    """One disc centred in an n x n cell, radius sqrt(vf * n^2 / pi) (Sec. 5.1 shape)."""
    c = (n - 1) / 2.0
    r = np.sqrt(vf * n * n / np.pi)
    y, x = np.mgrid[0:n, 0:n]
    return (((x - c) ** 2 + (y - c) ** 2) <= r * r).astype(np.uint8)


def centred_sphere(n: int, vf: float) -> np.ndarray:
    """One sphere centred in an n^3 cell, radius (3 vf n^3 / (4 pi))^(1/3) (Sec. 5.3 shape)."""
    c = (n - 1) / 2.0
    r = (3.0 * vf * n ** 3 / (4.0 * np.pi)) ** (1.0 / 3.0)
    z, y, x = np.ogrid[0:n, 0:n, 0:n]
    return (((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) <= r * r).astype(np.uint8)


def centred_annulus(n: int, vf: float, inner: float = 0.5) -> np.ndarray:
    """One ring centred in an n x n cell (Sec. 5.1, annular inclusion): inner radius = `inner`
    times the outer radius, ring area vf n^2."""
    c = (n - 1) / 2.0
    ro = np.sqrt(vf * n * n / (np.pi * (1.0 - inner * inner)))
    ri = inner * ro
    y, x = np.ogrid[0:n, 0:n]
    d2 = (x - c) ** 2 + (y - c) ** 2
    return ((d2 <= ro * ro) & (d2 > ri * ri)).astype(np.uint8)


def centred_ellipse(n: int, vf: float, aspect: float = 2.0) -> np.ndarray:
    """One ellipse centred in an n x n cell (Sec. 5.1, elliptical inclusion): semi-axis along x
    `aspect` times the one along y, area vf n^2."""
    c = (n - 1) / 2.0
    b = np.sqrt(vf * n * n / (np.pi * aspect))
    a = aspect * b
    y, x = np.ogrid[0:n, 0:n]
    return (((x - c) / a) ** 2 + ((y - c) / b) ** 2 <= 1.0).astype(np.uint8)


def centred_square(n: int, vf: float) -> np.ndarray:
    """One axis-aligned square centred in an n x n cell (Sec. 5.1, quadratic inclusion), side
    sqrt(vf) n."""
    c = (n - 1) / 2.0
    h = 0.5 * np.sqrt(vf) * n
    y, x = np.ogrid[0:n, 0:n]
    return ((np.abs(x - c) <= h) & (np.abs(y - c) <= h)).astype(np.uint8)


def laminate(shape: tuple, widths: tuple) -> np.ndarray:
    """Layers normal to x: phase p occupies widths[p] consecutive x columns, repeated."""
    nx = shape[-1]
    col = np.concatenate([np.full(w, p, np.uint8) for p, w in enumerate(widths)])
    reps = -(-nx // len(col))
    col = np.tile(col, reps)[:nx]
    return np.broadcast_to(col, shape).copy()


def _periodic_delta(a: np.ndarray, b: float, n: int) -> np.ndarray:
    d = np.abs(a - b)
    return np.minimum(d, n - d)


def _paint(phase: np.ndarray, centre, r: float) -> int:
    """Set voxels of one periodic disc/sphere to 1; returns the number newly set."""
    dim = phase.ndim
    n = phase.shape[0]
    lo = [int(np.floor(c - r)) for c in centre]
    hi = [int(np.ceil(c + r)) for c in centre]
    axes = [np.arange(l, h + 1) for l, h in zip(lo, hi)]
    if dim == 2:
        xs, ys = axes
        X, Y = np.meshgrid(xs, ys, indexing="xy")
        inside = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 <= r * r
        idx = (Y[inside] % n, X[inside] % n)
    else:
        xs, ys, zs = axes
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        inside = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2 <= r * r
        idx = (Z[inside] % n, Y[inside] % n, X[inside] % n)
    before = int(phase[idx].sum())
    phase[idx] = 1
    return int(len(idx[0])) - before


def _rsa(dim: int, n: int, r_range, vf: float, seed: int, gap: float = 1.0,
         max_attempts: int = 30000) -> np.ndarray:
    rng = _rng(seed)
    phase = np.zeros((n,) * dim, np.uint8)
    target = vf * phase.size
    centres = np.zeros((0, dim))
    radii = np.zeros(0)
    filled = 0
    attempts = 0
    while filled < target and attempts < max_attempts:
        attempts += 1
        c = rng.uniform(0.0, n, size=dim)
        r = rng.uniform(r_range[0], r_range[1])
        if len(radii):
            d2 = np.zeros(len(radii))
            for a in range(dim):
                d2 += _periodic_delta(centres[:, a], c[a], n) ** 2
            if np.any(np.sqrt(d2) < radii + r + gap):
                continue
        centres = np.vstack([centres, c])
        radii = np.append(radii, r)
        filled += _paint(phase, c, r)
    return phase


def random_discs(n: int, r_range=(8.0, 24.0), vf: float = 0.4, seed: int = 0) -> np.ndarray:
    """Periodic non-overlapping discs in an n x n cell (Sec. 5.2 style composite)."""
    return _rsa(2, n, r_range, vf, seed)


def random_spheres(n: int, r_range=(6.0, 12.0), vf: float = 0.25, seed: int = 0) -> np.ndarray:
    """Periodic non-overlapping spheres in an n^3 cell."""
    return _rsa(3, n, r_range, vf, seed)


def random_macro_strain(seed: int, dim: int, amplitude: float = 0.01) -> np.ndarray:
    """Symmetric macroscopic strain, entries U[-a, a], as the 6-vector (11,22,33,23,13,12).

    In 2D (plane strain) the out-of-plane entries 33, 23, 13 are zero.
    """
    rng = _rng(seed)
    v = rng.uniform(-amplitude, amplitude, size=6)
    if dim == 2:
        v[2] = v[3] = v[4] = 0.0
    return v
