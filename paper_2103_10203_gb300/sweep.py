"""Accuracy of reduced sets of frequencies against the full set (Sec. 5).

For a microstructure and a load (one macroscopic strain, or a load path), every ratio R and
every sampling pattern kind (the geometrically adapted pattern of Sec. 4.2, the fixed radial
pattern of Sec. 4.1) is solved on its reduced set and compared with the solve on the full set
of frequencies: the macroscopic error Ebar and the microscopic error E of Sec. 5, before and
after the compatibility step (Sec. 5.1). Patterns, solves, the compatibility step and the error
measures all run in the library's kernels; this module only strings the calls together.
"""

from __future__ import annotations

import math
import time

import numpy as np

from . import rf


def full_pattern(shape) -> np.ndarray:
    """Every frequency of a grid of shape (Ny, Nx) or (Nz, Ny, Nx), int32 [N, 3] (kx, ky, kz)."""
    sh = (1,) + tuple(shape) if len(shape) == 2 else tuple(shape)
    nz, ny, nx = sh
    kz, ky, kx = np.meshgrid(np.arange(nz) - (nz - 1) // 2, np.arange(ny) - (ny - 1) // 2,
                             np.arange(nx) - (nx - 1) // 2, indexing="ij")
    return np.stack([kx.ravel(), ky.ravel(), kz.ravel()], axis=1).astype(np.int32)


def pattern(kind: str, phase_map, k_target: int, inclusion_phase: int = 1, stream=None):
    if kind == "adapted":
        return rf.rf_pattern_adapted(phase_map, inclusion_phase, k_target, stream=stream)
    if kind == "radial":
        return rf.rf_pattern_radial(phase_map.shape, k_target, stream=stream)
    raise ValueError(kind)


def _run(solver, macro, path):
    t0 = time.perf_counter()
    if path is not None:
        out = solver.rf_solve_path(path)
        iters = int(np.sum(out["iters"]))
    else:
        out = solver.rf_solve(macro)
        iters = int(out["iters"])
    return iters, time.perf_counter() - t0


def pattern_study(phase_map, phases, ratios, macro=None, path=None,
                  kinds=("adapted", "radial"), inclusion_phase=1, tol=1e-6, max_iter=20000,
                  transform="fft", compat=True, stream=None):
    """Rows of (R, pattern kind) with K, update count, solve time and (Ebar, E) against the full
    set of frequencies, plus (Ebar, E) after the compatibility step when `compat` is set.
    Exactly one of `macro` (rf_solve) and `path` (rf_solve_path; errors at its last increment)
    is given. The radial pattern exists in 2D only. Returns (rows, reference summary)."""
    if (macro is None) == (path is None):
        raise ValueError("give exactly one of macro and path")
    pm = np.ascontiguousarray(phase_map, dtype=np.uint8)
    opts = dict(tol=tol, max_iter=max_iter, transform=transform)
    ref = rf.Solver(pm, phases, pattern=full_pattern(pm.shape), stream=stream, **opts)
    try:
        ref_iters, ref_s = _run(ref, macro, path)
        rows = []
        for R in ratios:
            K = int(math.ceil(R * pm.size - 1e-9))
            for kind in kinds:
                if kind == "radial" and pm.ndim != 2:
                    continue
                pat = pattern(kind, pm, K, inclusion_phase, stream)
                s = rf.Solver(pm, phases, pattern=pat, stream=stream, **opts)
                try:
                    iters, secs = _run(s, macro, path)
                    eb, e = s.rf_stress_errors(ref)
                    row = dict(ratio=R, pattern=kind, K=int(len(pat)), iters=iters,
                               solve_s=secs, Ebar=eb, E=e)
                    if compat:
                        s.rf_compat()     # the first call builds the full-set context
                        t0 = time.perf_counter()
                        s.rf_compat()
                        row["compat_s"] = time.perf_counter() - t0
                        row["Ebar_compat"], row["E_compat"] = s.rf_stress_errors(ref)
                    rows.append(row)
                finally:
                    s.close()
        return rows, dict(K=int(pm.size), iters=ref_iters, solve_s=ref_s)
    finally:
        ref.close()
