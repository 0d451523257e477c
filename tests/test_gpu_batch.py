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


@pytest.mark.parametrize("transform", ["dft", "fft"])
def test_batch_matches_single_solves(lib, transform):
    ph = elastic_phases()
    pms, pats, macros = population(14)
    b = lib.BatchSolver(pms, ph, pats, tol=1e-6, max_iter=2000, transform=transform)
    out = b.rf_batch_solve(macros)
    info = b.rf_batch_info()
    b.close()
    assert out["converged"] and np.all(out["status"] == 0)
    assert len(info["rows_per_item"]) == 5 and info["grid"] > 0
    # shared-memory FFT items of 1, 2, 4 or 8 rows, or warp-FFT items (rows of 64, 96, 128,
    # 192, 256 voxels: 85, 53, 42, 26, 21 rows)
    assert all(r in (1, 2, 4, 8, 85, 53, 42, 26, 21) for r in info["rows_per_item"])
    for i, (pm, pat) in enumerate(zip(pms, pats)):
        s = lib.Solver(pm, ph, pattern=pat, tol=1e-6, max_iter=2000)
        one = s.rf_solve(macros[i])
        s.close()
        assert abs(int(out["iters"][i]) - one["iters"]) <= 1, i
        assert rel(out["sigma_bar"][i], one["sigma_bar"]) <= 2e-6, i


@pytest.mark.parametrize("transform", ["dft", "fft"])
def test_batch_matches_oracle_at_fixed_update_counts(lib, transform):
    ph = elastic_phases()
    pms, pats, macros = population(9, seed0=300)
    b = lib.BatchSolver(pms, ph, pats, tol=0.0, max_iter=5, transform=transform)
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


def half_order(pat):
    """The batch's slot order of one RVE: pattern frequencies with kx >= 0, sorted by (kx, ky)."""
    return sorted((int(k[0]), int(k[1])) for k in pat if k[0] >= 0)


@pytest.mark.parametrize("transform,warps,resident", [("fft", -1, -1), ("fft", 2, -1),
                                                      ("dft", 0, -1), ("fft", 0, 1)])
def test_batch_reduced_coefficients_match_oracle_at_full_sizes(lib, transform, warps, resident):
    """Sides 64, 96, 128, 192 and 256 (the FE-FFT population's sizes: radix-2 and radix-3 FFT
    items along x and y, on shared memory (warps -1) or as warp-FFT row and column items with
    2, 3, 4, 6 and 8 points per lane (warps 2), or pruned-DFT items, or the RVE-resident solve
    (resident 1: a block per RVE for all its updates, the same warp-FFT transforms)), a fixed
    number of updates, every reduced strain coefficient compared with the oracle's (relative
    L2 per RVE <= 1e-5), and the homogenised stress (<= 1e-6)."""
    ph = elastic_phases()
    pms, pats, macros = [], [], []
    for i, side in enumerate((64, 96, 128, 192, 256)):
        c = make_config("c4", n=side, index=i)
        pms.append(c["phase_map"])
        pats.append(lib.rf_pattern_adapted(c["phase_map"], 1, c["k_target"]))
        macros.append(c["macro"])
    macros = np.array(macros)
    b = lib.BatchSolver(pms, ph, pats, tol=0.0, max_iter=4, transform=transform,
                        fft_row_warps=warps, batch_resident=resident)
    out = b.rf_batch_solve(macros)
    info = b.rf_batch_info()
    coeffs = b.rf_batch_reduced_strain().cpu().numpy()
    _, off = b.rf_batch_slots()
    b.close()
    assert np.all(out["iters"] == 4)
    assert info["resident"] == (resident > 0)
    if warps > 0:
        assert list(info["rows_per_item"]) == [85, 53, 42, 26, 21]
    elif transform == "fft":
        assert all(r in (1, 2, 4, 8) for r in info["rows_per_item"])
    for i, (pm, pat) in enumerate(zip(pms, pats)):
        r = O.solve(pm, ph, macros[i], pat, tol=0.0, max_iter=4)
        at = {(int(k[0]), int(k[1])): p for p, k in enumerate(pat)}
        hs = half_order(pat)
        assert off[i + 1] - off[i] == len(hs)
        want = np.array([[r.eps_hat[at[k], 0, 0], r.eps_hat[at[k], 1, 1], r.eps_hat[at[k], 0, 1]]
                         for k in hs])
        got = coeffs[off[i]:off[i + 1], :, 0] + 1j * coeffs[off[i]:off[i + 1], :, 1]
        assert rel(got, want) <= 1e-5, (i, rel(got, want))
        assert rel(out["sigma_bar"][i], r.sigma_bar) <= 1e-6, i


def test_batch_reports_divergence_and_non_finite_input(lib):
    """A reference medium from volume averages with a stiff minority phase (contrast 1000 at
    5 % volume) violates the contraction condition of the basic scheme: the measure grows by
    about 11x per update (the oracle shows it) and the RVE ends with RF_ERR_DIVERGED, while a
    homogeneous RVE beside it converges. A NaN macroscopic strain is rejected with
    RF_ERR_NONFINITE."""
    from synth import phase_table
    ph = phase_table([(1.0, 1.0, 0, 0, 0), (1000.0, 1000.0, 0, 0, 0)])
    good = np.zeros((32, 32), np.uint8)
    bad = np.zeros((32, 32), np.uint8)
    bad[10:17, 12:19] = 1                          # about 5 % stiff phase
    pats = [O.pattern_adapted(pm, 1, k_target(0.1, pm.size)) for pm in (good, bad)]
    macro = np.array([[0.01, 0, 0, 0, 0, 0.002]] * 2)
    r = O.solve(bad, ph, macro[1], pats[1], tol=0.0, max_iter=6, ref="volume",
                keep_history=True)
    assert r.history[-1] > 1e4 * min(r.history)
    b = lib.BatchSolver([good, bad], ph, pats, tol=1e-6, max_iter=500, ref="volume",
                        transform="fft")
    out = b.rf_batch_solve(macro)
    assert out["status"][0] == 0 and out["status"][1] == -4 and not out["converged"]
    assert out["iters"][1] < 20
    with pytest.raises(lib.RFError) as e:
        b.rf_batch_solve(np.array([[np.nan, 0, 0, 0, 0, 0], [0.01, 0, 0, 0, 0, 0]]))
    assert e.value.code == -3
    b.close()
    s = lib.Solver(bad, ph, pattern=pats[1], tol=1e-6, max_iter=500, ref="volume")
    with pytest.raises(lib.RFError) as e:
        s.rf_solve(macro[1])
    assert e.value.code == -4
    s.close()


def c4_population(n, seed_index=0):
    pms, pats, macros = [], [], []
    for i in range(n):
        side = (64, 96, 128, 192, 256)[i % 5]
        c = make_config("c4", n=side, index=seed_index + i)
        pms.append(c["phase_map"])
        pats.append(O.pattern_adapted(c["phase_map"], 1, c["k_target"]))
        macros.append(c["macro"])
    return pms, pats, np.array(macros)


def test_batch_resident_solve_matches_sweeps(lib):
    """The RVE-resident solve against the sweep kernels on the same 10 RVEs (sides 64 to 256):
    the same updates and convergence rules, so iteration counts within one and homogenised
    stresses within 2e-6; a warm start from the converged coefficients (device export mapped
    to the host warm layout) converges in at most 2 updates; a re-solve repeats the first."""
    ph = elastic_phases()
    pms, pats, macros = c4_population(10, seed_index=70)
    sw = lib.BatchSolver(pms, ph, pats, tol=1e-6, max_iter=500, transform="fft",
                         batch_resident=-1)
    ref = sw.rf_batch_solve(macros)
    assert not sw.rf_batch_info()["resident"]
    sw.close()
    b = lib.BatchSolver(pms, ph, pats, tol=1e-6, max_iter=500, transform="fft",
                        batch_resident=1)
    assert b.rf_batch_info()["resident"]
    out = b.rf_batch_solve(macros)
    assert out["converged"] and np.all(out["status"] == 0)
    assert np.all(np.abs(out["iters"].astype(int) - ref["iters"].astype(int)) <= 1)
    for i in range(len(pms)):
        assert rel(out["sigma_bar"][i], ref["sigma_bar"][i]) <= 2e-6, i
    coeffs = b.rf_batch_reduced_strain().cpu().numpy()
    _, off = b.rf_batch_slots()
    warm = []
    for i, pat in enumerate(pats):
        at = {k: p for p, k in enumerate(half_order(pat))}
        w = np.zeros((len(pat), 6, 2), np.float32)
        for p, k in enumerate(pat):
            key = (int(k[0]), int(k[1]))
            if key in at:
                c = coeffs[off[i] + at[key]]
                for a, comp in ((0, 0), (1, 1), (5, 2)):   # Voigt 11, 22, 12
                    w[p, a] = c[comp]
        warm.append(w if i % 2 == 0 else None)
    hot = b.rf_batch_solve(macros, warm=warm)
    again = b.rf_batch_solve(macros)
    b.close()
    for i in range(len(pms)):
        if warm[i] is not None:
            assert hot["iters"][i] <= 2 < out["iters"][i], i
        else:
            assert hot["iters"][i] == out["iters"][i], i
        assert rel(hot["sigma_bar"][i], out["sigma_bar"][i]) <= 2e-6, i
    assert np.array_equal(again["sigma_bar"], out["sigma_bar"])
    assert np.array_equal(again["iters"], out["iters"])


def test_batch_resident_mode_selection(lib):
    """batch_resident: 1 where every RVE is square with a warp-FFT side, else the sweeps; -1
    never; values outside -1..1 are rejected; the DFT transform never runs resident."""
    ph = elastic_phases()
    pms, pats, macros = c4_population(3, seed_index=90)
    for opt, want in ((1, True), (-1, False)):
        b = lib.BatchSolver(pms, ph, pats, tol=1e-6, max_iter=50, transform="fft",
                            batch_resident=opt)
        assert b.rf_batch_info()["resident"] == want
        b.close()
    b = lib.BatchSolver(pms, ph, pats, tol=1e-6, max_iter=50, transform="dft", batch_resident=1)
    assert not b.rf_batch_info()["resident"]
    b.close()
    small, spats, _ = population(2)                     # sides 16 and 24: not eligible
    b = lib.BatchSolver(small + pms, ph, spats + pats, tol=1e-6, max_iter=50, transform="fft",
                        batch_resident=1)
    assert not b.rf_batch_info()["resident"]
    b.close()
    with pytest.raises(lib.RFError):
        lib.BatchSolver(pms, ph, pats, transform="fft", batch_resident=2)


def test_batch_resident_reports_divergence(lib):
    """The RVE-resident solve applies the same divergence rule per RVE: a stiff minority phase
    (contrast 1000 at about 5 % volume) with a volume-average reference medium ends with
    RF_ERR_DIVERGED within a few updates, while the homogeneous RVE beside it converges."""
    from synth import phase_table
    ph = phase_table([(1.0, 1.0, 0, 0, 0), (1000.0, 1000.0, 0, 0, 0)])
    good = np.zeros((64, 64), np.uint8)
    bad = np.zeros((64, 64), np.uint8)
    bad[20:34, 24:38] = 1                          # 196 of 4096 voxels
    pats = [O.pattern_adapted(pm, 1, k_target(0.1, pm.size)) for pm in (good, bad)]
    macro = np.array([[0.01, 0, 0, 0, 0, 0.002]] * 2)
    b = lib.BatchSolver([good, bad], ph, pats, tol=1e-6, max_iter=500, ref="volume",
                        transform="fft", batch_resident=1)
    assert b.rf_batch_info()["resident"]
    out = b.rf_batch_solve(macro)
    b.close()
    assert out["status"][0] == 0 and out["status"][1] == -4 and not out["converged"]
    assert out["iters"][1] < 20
