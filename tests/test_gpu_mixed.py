"""Mixed macroscopic stress/strain control (FE-FFT Gauss-point coupling, Sec. 1) through the C ABI
against the oracle's mixed control, element by element at equal update counts (strain field and
macroscopic strain <= 1e-5 relative L2, homogenised stress <= 1e-6), in every transform mode."""

import numpy as np
import pytest

import oracle as O
from oracle.rf_oracle import VOIGT
from synth import random_discs, random_spheres
from synth.configs import elastic_phases, j2_phases, k_target

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))


def vec6_field(t):
    g = t[0] if t.shape[0] == 1 else t
    return np.stack([g[..., i, j] for (i, j) in VOIGT])


MODES = [dict(transform="dft"), dict(transform="fft", fft_fuse=-1),
         dict(transform="fft", fft_fuse=1), dict(transform="fft", fft_fuse=2),
         dict(transform="fft", fft_fuse=3)]


@pytest.mark.parametrize("mode", range(len(MODES)))
def test_mixed_control_2d_matches_oracle(lib, mode):
    pm = random_discs(64, (4.0, 9.0), 0.4, seed=2)
    ph = elastic_phases()
    pat = O.pattern_adapted(pm, 1, k_target(0.05, pm.size))
    control = [1, 0, 0, 0, 0, 1]                      # sigma_11, sigma_12 prescribed
    target = np.array([0.5, -0.002, 0, 0, 0, 0.05])
    s = lib.Solver(pm, ph, pattern=pat, tol=0.0, max_iter=8, **MODES[mode])
    out = s.rf_solve_mixed(control, target)
    eps, _, _ = s.rf_get_fields()
    s.close()
    r = O.solve(pm, ph, target, pat, tol=0.0, max_iter=8, control=control)
    assert rel(eps, vec6_field(r.eps)) <= 1e-5
    assert rel(out["sigma_bar"], r.sigma_bar) <= 1e-6
    assert rel(out["strain_bar"], r.macro_strain) <= 1e-5


@pytest.mark.parametrize("transform", ["dft", "fft"])
def test_mixed_control_3d_matches_oracle(lib, transform):
    pm = random_spheres(16, (2.0, 4.0), 0.25, seed=3)
    ph = elastic_phases()
    pat = O.pattern_adapted(pm, 1, 410)
    control = [0, 1, 1, 0, 1, 0]
    target = np.array([0.01, 0.2, 0.0, 0.001, -0.03, 0.0])
    s = lib.Solver(pm, ph, pattern=pat, tol=0.0, max_iter=6, transform=transform)
    out = s.rf_solve_mixed(control, target)
    eps, _, _ = s.rf_get_fields()
    s.close()
    r = O.solve(pm, ph, target, pat, tol=0.0, max_iter=6, control=control)
    assert rel(eps, vec6_field(r.eps)) <= 1e-5
    assert rel(out["sigma_bar"], r.sigma_bar) <= 1e-6
    assert rel(out["strain_bar"], r.macro_strain) <= 1e-5


def test_mixed_control_j2_load_path_matches_oracle(lib):
    """Plane-strain loading in eps_11 with sigma_22 = 0 prescribed (the transverse direction
    free), J2 matrix, three increments into the plastic range with commits."""
    pm = random_discs(64, (4.0, 9.0), 0.4, seed=2)
    ph = j2_phases()
    pat = O.pattern_adapted(pm, 1, k_target(0.05, pm.size))
    control = [0, 1, 0, 0, 0, 0]
    path = np.zeros((3, 6))
    path[:, 0] = [0.005, 0.01, 0.015]
    s = lib.Solver(pm, ph, pattern=pat, tol=0.0, max_iter=6, transform="fft")
    out = s.rf_solve_path_mixed(control, path)
    eps, _, alpha = s.rf_get_fields()
    s.close()
    sbar, _, r = O.solve_path(pm, ph, path, pat, fixed_iters=[6, 6, 6], control=control)
    for n in range(3):
        assert rel(out["sigma_bar"][n], sbar[n]) <= 1e-6, n
    assert rel(out["strain_bar"][-1], r.macro_strain) <= 1e-5
    assert rel(eps, vec6_field(r.eps)) <= 1e-5
    assert alpha.max() > 0


def test_mixed_control_reaches_its_stress_targets(lib):
    """Solved to the tolerance, the prescribed average stresses hold and a strain-controlled solve
    at the reached macro strain gives the same homogenised stress."""
    pm = random_discs(64, (4.0, 9.0), 0.4, seed=5)
    ph = elastic_phases()
    pat = lib.rf_pattern_adapted(pm, 1, k_target(0.05, pm.size))
    control = [1, 1, 0, 0, 0, 0]
    target = np.array([0.3, -0.1, 0, 0, 0, 0.0])
    s = lib.Solver(pm, ph, pattern=pat, tol=1e-7, max_iter=5000, transform="fft")
    out = s.rf_solve_mixed(control, target)
    plain = s.rf_solve(out["strain_bar"])
    s.close()
    assert out["converged"]
    assert abs(out["sigma_bar"][0] - 0.3) <= 1e-5 * 0.3 and abs(out["sigma_bar"][1] + 0.1) <= 1e-5
    assert rel(plain["sigma_bar"], out["sigma_bar"]) <= 1e-5


def test_mixed_control_argument_checks(lib):
    pm = random_discs(32, (3.0, 5.0), 0.3, seed=1)
    s = lib.Solver(pm, elastic_phases(), pattern=O.pattern_adapted(pm, 1, 51))
    with pytest.raises(lib.RFError) as e:
        s.rf_solve_mixed([0, 0, 1, 0, 0, 0], np.zeros(6))     # 2D: sigma_33 cannot be a target
    assert e.value.code == -1
    with pytest.raises(lib.RFError) as e:
        s.rf_solve_mixed([2, 0, 0, 0, 0, 0], np.zeros(6))
    assert e.value.code == -1
    with pytest.raises(lib.RFError) as e:
        s.rf_solve_mixed([1, 0, 0, 0, 0, 0], np.array([np.nan, 0, 0, 0, 0, 0]))
    assert e.value.code == -3
    s.close()
