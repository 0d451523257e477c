"""Compatibility step (Sec. 5.1: the Lippmann-Schwinger equation solved once on the full set of
frequencies from the reduced solution) through the C ABI, against the oracle's `compat`.

The reduced solves run a fixed number of updates so that the oracle replays exactly the same
reduced solution; the step's strain and stress fields are compared with relative L2 <= 1e-5 and
the homogenised stress with <= 1e-6 (FP32 against FP64, as every parity test here)."""

import numpy as np
import pytest

import oracle as O
from oracle.rf_oracle import VOIGT
from synth import centred_disc, random_discs, random_macro_strain, random_spheres
from synth.configs import elastic_phases, j2_phases, k_target, uniaxial_path

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))


def vec6_field(t):
    g = t[0] if t.shape[0] == 1 else t
    return np.stack([g[..., i, j] for (i, j) in VOIGT])


CASES = {
    # name: (phase map, phases, macro, K, transform of the reduced solve)
    "disc64_fft": (centred_disc(64, 0.3), elastic_phases(), np.array([0.01, -0.01, 0, 0, 0, 0]),
                   205, "fft"),
    "discs48_dft": (random_discs(48, (3.0, 7.0), 0.4, seed=9), elastic_phases(),
                    random_macro_strain(4, 2), 116, "dft"),
    "odd_21x15": (random_discs(21, (2.0, 4.0), 0.3, seed=9)[:, :15].copy(), elastic_phases(),
                  random_macro_strain(8, 2), 64, "dft"),
    "spheres16": (random_spheres(16, (2.0, 4.0), 0.25, seed=3), elastic_phases(),
                  random_macro_strain(30, 3), 164, "fft"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_compat_step_matches_oracle(lib, name):
    pm, ph, macro, K, transform = CASES[name]
    pat = O.pattern_adapted(pm, 1, K)
    s = lib.Solver(pm, ph, pattern=pat, tol=0.0, max_iter=8, transform=transform)
    red = s.rf_solve(macro)
    sbar = s.rf_compat()
    eps, sig, _ = s.rf_get_fields()
    again = s.rf_compat()                    # the reduced solution is unchanged by the step
    s.close()
    r = O.solve(pm, ph, macro, pat, tol=0.0, max_iter=8)
    eps_c, sig_c, sbar_c = O.compat(pm, ph, r.eps, macro)
    assert rel(eps, vec6_field(eps_c)) <= 1e-5
    assert rel(sig, vec6_field(sig_c)) <= 1e-5
    assert rel(sbar, sbar_c) <= 1e-6
    assert np.array_equal(again, sbar)
    assert rel(red["sigma_bar"], r.sigma_bar) <= 1e-6


def test_compat_step_after_a_j2_load_path(lib):
    """After three increments into the plastic range with commits, the step uses the committed
    internal variables."""
    pm = random_discs(64, (4.0, 9.0), 0.4, seed=2)
    ph = j2_phases()
    pat = O.pattern_adapted(pm, 1, k_target(0.05, pm.size))
    path = uniaxial_path(20, 0.02)[[4, 9, 14]]
    s = lib.Solver(pm, ph, pattern=pat, tol=0.0, max_iter=6, transform="fft")
    s.rf_solve_path(path)
    sbar = s.rf_compat()
    eps, sig, alpha = s.rf_get_fields()
    s.close()
    _, _, r = O.solve_path(pm, ph, path, pat, fixed_iters=[6, 6, 6])
    eps_c, sig_c, sbar_c = O.compat(pm, ph, r.eps, path[-1], eps_p=r.eps_p, alpha=r.alpha)
    assert rel(eps, vec6_field(eps_c)) <= 1e-5
    assert rel(sig, vec6_field(sig_c)) <= 1e-5
    assert rel(sbar, sbar_c) <= 1e-6
    assert alpha.max() > 0


def test_compat_step_needs_a_solve(lib):
    pm = centred_disc(16, 0.3)
    s = lib.Solver(pm, elastic_phases(), pattern=O.pattern_adapted(pm, 1, 13))
    with pytest.raises(lib.RFError) as e:
        s.rf_compat()
    assert e.value.code == -7
    s.close()
