"""Trends the paper reports for reduced sets of frequencies (Sec. 5.1, 5.2), checked with the
oracle on small cells of the paper-shaped inputs (CPU only). These are trends, not values: the
paper's geometries exist only as figures, so no number of its error plots is reproduced.

* The geometrically adapted pattern gives smaller macroscopic and microscopic stress errors
  than the fixed radial pattern at small R (Sec. 5.1: one inclusion of four shapes; Sec. 5.2:
  several inclusions).
* The errors of the adapted pattern shrink as R grows and vanish on the full set.
* The compatibility step (Sec. 5.1) lowers the microscopic error of the adapted solution.
"""

import numpy as np
import pytest

import oracle as O
from synth import make_config
from synth.configs import k_target

RATIOS = (0.0154, 0.0306, 0.0602)


def _errors(pm, ph, macro, pat, ref):
    r = O.solve(pm, ph, macro, pat, tol=1e-8)
    return O.errors(r.sigma, ref.sigma, r.sigma_bar, ref.sigma_bar), r


@pytest.mark.parametrize("case", ["circle", "annulus", "ellipse", "square", "several"])
def test_adapted_pattern_beats_radial_and_converges_to_the_full_set(case):
    c = make_config("p52", n=32) if case == "several" else make_config("p51", n=32, shape=case)
    pm, ph, macro = c["phase_map"], c["phases"], c["macro"]
    full = O.full_pattern((1,) + pm.shape)
    ref = O.solve(pm, ph, macro, full, tol=1e-10)
    adapted = []
    for R in RATIOS:
        K = k_target(R, pm.size)
        (eb_a, e_a), r = _errors(pm, ph, macro, O.pattern_adapted(pm, 1, K), ref)
        (eb_r, e_r), _ = _errors(pm, ph, macro, O.pattern_radial(pm.shape, K), ref)
        assert eb_a < eb_r and e_a < e_r, (R, eb_a, eb_r, e_a, e_r)
        adapted.append((eb_a, e_a))
        _, sc, sbc = O.compat(pm, ph, r.eps, macro)
        assert O.errors(sc, ref.sigma, sbc, ref.sigma_bar)[1] < e_a
    eb, e = np.array(adapted).T
    assert np.all(np.diff(eb) < 0) and np.all(np.diff(e) < 0)
    (eb_f, e_f), _ = _errors(pm, ph, macro, O.pattern_adapted(pm, 1, pm.size), ref)
    assert eb_f < 1e-8 and e_f < 1e-8
