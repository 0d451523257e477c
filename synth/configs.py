"""The five synthetic workloads (sizes, moduli, seeds) and a builder for each.

c1  2D 64^2, one centred circular fibre (vf 0.3), elastic, eps_11 = 0.01, K = 5 %.
c2  2D 1024^2, random discs r in [8, 24], vf 0.4, J2 matrix (sigma_y0 0.25 GPa, H 1 GPa),
    20 uniaxial-strain increments of eps_11 to 0.02, K in {1, 5, 10} %.
c3  3D 128^3, random spheres r in [6, 12], vf 0.25, elastic, random symmetric strain, K = 2 %.
c4  batch of 2D RVEs with sides in {64, 96, 128, 192, 256}, vf in [0.2, 0.5], K = 5 %.
c5  2D 128^2 fibre RVEs (vf in [0.2, 0.5], radius 8-24), K = 5 %, for the warm-start network.

Inputs shaped like the paper's own examples (Sec. 5; the geometries exist only as figures, so
sizes of the inclusions are readings), with the paper's moduli lambda_I = mu_I = 2 GPa,
lambda_M = mu_M = 1 GPa:
p51   2D 256^2, one centred inclusion: circle, annulus, ellipse or square (vf 0.3),
      ebar_11 = 0.01, ebar_22 = -0.01 (Sec. 5.1).
p52   2D 256^2, several circular inclusions (r 16-32, vf 0.3, seed 52), elastic, or with a J2
      matrix (H = 0.01 GPa, sigma_y0 = 0.01 GPa) loaded in 100 equal increments to
      ebar = [[0.01, 0.002], [0.002, -0.01]] (Sec. 5.2).
p53   3D 256^3, one centred sphere (vf 0.3), elastic, ebar_11 = 0.01 (Sec. 5.3).
"""

from __future__ import annotations

import math

import numpy as np

from .materials import lame, phase_table
from .microstructure import (centred_annulus, centred_disc, centred_ellipse, centred_sphere,
                             centred_square, random_discs, random_macro_strain, random_spheres)

MATRIX_E, MATRIX_NU = 70.0, 0.3
FIBRE_E, FIBRE_NU = 400.0, 0.2
YIELD, HARDENING = 0.25, 1.0


def k_target(ratio: float, n_vox: int) -> int:
    """ceil(R * N) frequencies, with a guard against the binary representation of R."""
    return int(math.ceil(ratio * n_vox - 1e-9))


def elastic_phases():
    lm, mm = lame(MATRIX_E, MATRIX_NU)
    lf, mf = lame(FIBRE_E, FIBRE_NU)
    return phase_table([(lm, mm, 0.0, 0.0, 0), (lf, mf, 0.0, 0.0, 0)])


def j2_phases():
    lm, mm = lame(MATRIX_E, MATRIX_NU)
    lf, mf = lame(FIBRE_E, FIBRE_NU)
    return phase_table([(lm, mm, YIELD, HARDENING, 1), (lf, mf, 0.0, 0.0, 0)])


PAPER_INCLUSION = (2.0, 2.0)    # lambda_I, mu_I (GPa), Sec. 5.1-5.3
PAPER_MATRIX = (1.0, 1.0)       # lambda_M, mu_M
PAPER_YIELD, PAPER_HARDENING = 0.01, 0.01   # Sec. 5.2 elastoplastic matrix


def paper_phases(plastic: bool = False):
    """Phase 0 = matrix, phase 1 = inclusion, with the moduli of the paper's examples."""
    lm, mm = PAPER_MATRIX
    li, mi = PAPER_INCLUSION
    if plastic:
        return phase_table([(lm, mm, PAPER_YIELD, PAPER_HARDENING, 1), (li, mi, 0.0, 0.0, 0)])
    return phase_table([(lm, mm, 0.0, 0.0, 0), (li, mi, 0.0, 0.0, 0)])


SHAPES_51 = {"circle": centred_disc, "annulus": centred_annulus, "ellipse": centred_ellipse,
             "square": centred_square}

CONFIGS = {
    "c1": dict(dim=2, n=64, vf=0.3, ratio=0.05, plastic=False),
    "c2": dict(dim=2, n=1024, vf=0.4, r_range=(8.0, 24.0), seed=2, ratios=(0.01, 0.05, 0.10),
               plastic=True, n_steps=20, final_strain=0.02),
    "c3": dict(dim=3, n=128, vf=0.25, r_range=(6.0, 12.0), seed=3, strain_seed=30, ratio=0.02,
               plastic=False),
    "c4": dict(dim=2, sides=(64, 96, 128, 192, 256), vf_range=(0.2, 0.5), r_range=(8.0, 24.0),
               seed0=40000, ratio=0.05, plastic=False),
    "c5": dict(dim=2, n=128, vf_range=(0.2, 0.5), r_range=(8.0, 24.0), ratio=0.05,
               train_seed0=500000, test_seed0=900000, plastic=False),
    "p51": dict(dim=2, n=256, vf=0.3, ratio=0.0154),
    "p52": dict(dim=2, n=256, vf=0.3, r_range=(16.0, 32.0), seed=52, ratio=0.0154, n_steps=100),
    "p53": dict(dim=3, n=256, vf=0.3, ratio=0.0154),
}

# the paper's percentages of frequencies R (the rows of its timing tables, Sec. 5)
PAPER_RATIOS = (0.0154, 0.0306, 0.0602, 0.1164, 0.2166, 0.3679)


def uniaxial_path(n_steps: int, final: float) -> np.ndarray:
    """n_steps equal increments of eps_11 up to `final`, other components 0: [n_steps, 6]."""
    path = np.zeros((n_steps, 6))
    path[:, 0] = final * np.arange(1, n_steps + 1) / n_steps
    return path


def make_config(name: str, n: int | None = None, index: int = 0, shape: str = "circle",
                plastic: bool = False) -> dict:
    """Build phase map, phase table, macro strain(s) and K target for one workload.

    `n` overrides the grid side (scaled-down parity cases); `index` picks one RVE of the
    batch/training populations (c4, c5); `shape` picks the p51 inclusion; `plastic` the p52
    elastoplastic matrix and load path.
    """
    cfg = CONFIGS[name]
    out = dict(name=name, dim=cfg["dim"])
    if name == "c1":
        side = n or cfg["n"]
        out["phase_map"] = centred_disc(side, cfg["vf"])
        out["phases"] = elastic_phases()
        out["macro"] = np.array([0.01, 0, 0, 0, 0, 0], float)
        out["ratio"] = cfg["ratio"]
    elif name == "c2":
        side = n or cfg["n"]
        scale = side / cfg["n"]
        rr = (max(1.5, cfg["r_range"][0] * scale), max(2.0, cfg["r_range"][1] * scale))
        out["phase_map"] = random_discs(side, rr, cfg["vf"], cfg["seed"])
        out["phases"] = j2_phases()
        out["path"] = uniaxial_path(cfg["n_steps"], cfg["final_strain"])
        out["macro"] = out["path"][-1]
        out["ratio"] = 0.05
        out["ratios"] = cfg["ratios"]
    elif name == "c3":
        side = n or cfg["n"]
        scale = side / cfg["n"]
        rr = (max(1.5, cfg["r_range"][0] * scale), max(2.0, cfg["r_range"][1] * scale))
        out["phase_map"] = random_spheres(side, rr, cfg["vf"], cfg["seed"])
        out["phases"] = elastic_phases()
        out["macro"] = random_macro_strain(cfg["strain_seed"], 3)
        out["ratio"] = cfg["ratio"]
    elif name == "c4":
        seed = cfg["seed0"] + index
        rng = np.random.Generator(np.random.PCG64(seed))
        side = n or int(rng.choice(cfg["sides"]))
        vf = float(rng.uniform(*cfg["vf_range"]))
        out["phase_map"] = random_discs(side, cfg["r_range"], vf, seed)
        out["phases"] = elastic_phases()
        out["macro"] = random_macro_strain(seed + 1, 2)
        out["ratio"] = cfg["ratio"]
    elif name == "c5":
        seed = index
        rng = np.random.Generator(np.random.PCG64(seed))
        side = n or cfg["n"]
        vf = float(rng.uniform(*cfg["vf_range"]))
        out["phase_map"] = random_discs(side, cfg["r_range"], vf, seed)
        out["phases"] = elastic_phases()
        out["macro"] = random_macro_strain(seed + 1, 2)
        out["ratio"] = cfg["ratio"]
    elif name == "p51":
        side = n or cfg["n"]
        out["phase_map"] = SHAPES_51[shape](side, cfg["vf"])
        out["phases"] = paper_phases()
        out["macro"] = np.array([0.01, -0.01, 0, 0, 0, 0], float)
        out["ratio"] = cfg["ratio"]
    elif name == "p52":
        side = n or cfg["n"]
        scale = side / cfg["n"]
        rr = (max(1.5, cfg["r_range"][0] * scale), max(2.0, cfg["r_range"][1] * scale))
        out["phase_map"] = random_discs(side, rr, cfg["vf"], cfg["seed"])
        out["phases"] = paper_phases(plastic)
        out["macro"] = np.array([0.01, -0.01, 0, 0, 0, 0.002], float)
        steps = cfg["n_steps"]
        out["path"] = out["macro"][None, :] * (np.arange(1, steps + 1) / steps)[:, None]
        out["ratio"] = cfg["ratio"]
    elif name == "p53":
        side = n or cfg["n"]
        out["phase_map"] = centred_sphere(side, cfg["vf"])
        out["phases"] = paper_phases()
        out["macro"] = np.array([0.01, 0, 0, 0, 0, 0], float)
        out["ratio"] = cfg["ratio"]
    else:
        raise KeyError(name)
    out["k_target"] = k_target(out["ratio"], out["phase_map"].size)
    return out
