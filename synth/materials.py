"""Material constants of the synthetic workloads (GPa throughout)."""

from __future__ import annotations

import numpy as np

# phase record: lambda, mu, sigma_y0, hardening H, plastic flag
PHASE_DTYPE = np.dtype([("lam", "f8"), ("mu", "f8"), ("sigma_y0", "f8"),
                        ("hardening", "f8"), ("plastic", "i4"), ("_pad", "i4")])


def lame(E: float, nu: float) -> tuple:
    """(lambda, mu) from Young's modulus and Poisson's ratio (3D isotropic relations)."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def phase_table(rows) -> np.ndarray:
    """rows: iterable of (lambda, mu, sigma_y0, H, plastic) -> structured array."""
    out = np.zeros(len(rows), PHASE_DTYPE)
    for i, r in enumerate(rows):
        out[i] = (r[0], r[1], r[2], r[3], int(r[4]), 0)
    return out
