"""Batched solve of many RVEs of uneven size (persistent kernels over work lists) against
single-RVE solves and the FP64 oracle."""

import numpy as np
import pytest

import oracle as O
from oracle.rf_oracle import VOIGT
from synth import make_config, random_discs, random_macro_strain
from synth.configs import elastic_phases, k_target

pytestmark = pytest.mark.gpu


def population(n, sides=(16, 24, 32, 48, 20), seed0=100):
    pms, pats, macros = [], [], []
    for i in range(n):
        side = sides[i % len(sides)]
        rng = np.random.default_rng(seed0 + i)
        vf = float(rng.uniform(0.2, 0.45))
        pm = random_discs(side, (2.0, max(3.0, side / 6)), vf, seed=seed0 + i)
        if i % 7 == 3:   # a rectangular cell
            pm = np.ascontiguousarray(pm[: side // 2 + 2])
        pms.append(pm)
        pats.append(O.pattern_adapted(pm, 1, k_target(0.08, pm.size)))
        macros.append(random_macro_strain(seed0 + 1000 + i, 2))
    return pms, pats, np.array(macros)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))


def test_batch_matches_single_solves(lib):
    ph = elastic_phases()
    pms, pats, macros = population(14)
    b = lib.BatchSolver(pms, ph, pats, tol=1e-6, max_iter=2000)
    out = b.rf_batch_solve(macros)
    info = b.rf_batch_info()
    b.close()
    assert out["converged"] and np.all(out["status"] == 0)
    assert info["rows_per_item"] in (1, 2, 4, 8) and info["grid"] > 0
    for i, (pm, pat) in enumerate(zip(pms, pats)):
        s = lib.Solver(pm, ph, pattern=pat, tol=1e-6, max_iter=2000)
        one = s.rf_solve(macros[i])
        s.close()
        assert abs(int(out["iters"][i]) - one["iters"]) <= 1, i
        assert rel(out["sigma_bar"][i], one["sigma_bar"]) <= 2e-6, i


def test_batch_matches_oracle_at_fixed_update_counts(lib):
    ph = elastic_phases()
    pms, pats, macros = population(9, seed0=300)
    b = lib.BatchSolver(pms, ph, pats, tol=0.0, max_iter=5)
    out = b.rf_batch_solve(macros)
    b.close()
    assert np.all(out["iters"] == 5) and np.all(out["status"] == 1)
    for i, (pm, pat) in enumerate(zip(pms, pats)):
        r = O.solve(pm, ph, macros[i], pat, tol=0.0, max_iter=5)
        assert rel(out["sigma_bar"][i], r.sigma_bar) <= 1e-6, i
        assert abs(out["residuals"][i] - r.residual) <= 1e-4 * r.residual, i


def test_batch_warm_start_and_resolve(lib):
    ph = elastic_phases()
    pms, pats, macros = population(6, seed0=500)
    warm = []
    for i, (pm, pat) in enumerate(zip(pms, pats)):
        r = O.solve(pm, ph, macros[i], pat, tol=1e-9, max_iter=3000)
        w = np.zeros((len(pat), 6, 2), np.float32)
        for a, (p, q) in enumerate(VOIGT):
            w[:, a, 0] = r.eps_hat[:, p, q].real
            w[:, a, 1] = r.eps_hat[:, p, q].imag
        warm.append(w if i % 2 == 0 else None)     # half the RVEs start cold
    b = lib.BatchSolver(pms, ph, pats, tol=1e-6, max_iter=2000)
    cold = b.rf_batch_solve(macros)
    hot = b.rf_batch_solve(macros, warm=warm)
    again = b.rf_batch_solve(macros)                # re-solve reuses the captured graphs
    b.close()
    for i in range(len(pms)):
        if warm[i] is not None:
            assert hot["iters"][i] <= 2 < cold["iters"][i]
        else:
            assert hot["iters"][i] == cold["iters"][i]
        assert rel(hot["sigma_bar"][i], cold["sigma_bar"][i]) <= 2e-6
    assert np.array_equal(again["sigma_bar"], cold["sigma_bar"])


def test_batch_rejects_plastic_phases_and_bad_patterns(lib):
    from synth.configs import j2_phases
    pms, pats, _ = population(2)
    with pytest.raises(lib.RFError):
        lib.BatchSolver(pms, j2_phases(), pats)
    bad = [pats[0][1:], pats[1]]
    with pytest.raises(lib.RFError):
        lib.BatchSolver(pms, elastic_phases(), bad)
