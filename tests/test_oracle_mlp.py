"""Pins of the warm-start network oracle: GELU against its table value and derivative, the
harmonics against trigonometry, the head against the scheme's first update (Born term, Sec. 4
step c on the plain start), gradients against central finite differences, Adam against a
hand-worked step, descriptors against symmetry and sum rules, and the premise of the head
(the elastic fixed point is linear in ebar) against the scheme itself."""

import math

import numpy as np

import oracle as O
from oracle import mlp
from oracle.rf_oracle import green_operator, isotropic_stiffness, wave_vector
from synth import centred_disc, laminate, random_discs
from synth.configs import elastic_phases


def test_gelu_values_and_derivative():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    # GELU(1) = Phi(1) = 0.8413447460685429 (standard normal CDF table value)
    assert np.isclose(mlp.gelu(np.array([1.0]))[0], 0.8413447460685429, rtol=1e-14)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert np.isclose(mlp.gelu(np.array([-1.0]))[0], -(1 - 0.8413447460685429), rtol=1e-13)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, atol=1e-8)


def test_harmonics_and_basis_layout():
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal(50), rng.standard_normal(50)
    t = np.arctan2(b, a)
    h = mlp.harmonics(a, b)
    want = [np.ones(50)]
    for m in (2, 4, 6, 8):
        want += [np.cos(m * t), np.sin(m * t)]
    assert np.allclose(h, np.array(want), atol=1e-12)
    phi = mlp.basis(a, b)
    rho = np.hypot(a, b) / mlp.RHO_REF
    assert np.allclose(phi[:9], h) and np.allclose(phi[9:18], h * rho)
    assert np.allclose(phi[18:], h * rho ** 2)


def _first_update_transfer(n1, n2, lam0, mu0):
    """-Gamma^(n) : (C_f - C_m) : E_d, components (11, 22, 12), continuous operator."""
    ph = elastic_phases()
    dC = isotropic_stiffness(ph[1]["lam"] - ph[0]["lam"], ph[1]["mu"] - ph[0]["mu"])
    q = np.zeros((len(n1), 3))
    q[:, 0], q[:, 1] = n1, n2
    G = green_operator(q, lam0, mu0)
    E = np.zeros((3, 3, 3))
    E[0, 0, 0] = 1
    E[1, 1, 1] = 1
    E[2, 0, 1] = E[2, 1, 0] = 1
    T = -np.einsum("kijab,abcd,ecd->kije", G, dC, E)
    return np.stack([T[:, 0, 0, :], T[:, 1, 1, :], T[:, 0, 1, :]], axis=1)   # [n, c, d]


def test_head_reproduces_the_first_update():
    """Fit the 27-term expansion to the Born transfer of one geometry, then the head with those
    coefficients must give the scheme's first update on ANOTHER geometry and macro strain
    exactly (the transfer depends on the direction of k only, degree 4 in it)."""
    ph = elastic_phases()
    pmA = random_discs(24, (2.0, 5.0), 0.3, seed=1)
    patA = O.pattern_adapted(pmA, 1, 120)
    lam0 = 0.5 * (ph[0]["lam"] + ph[1]["lam"])
    mu0 = 0.5 * (ph[0]["mu"] + ph[1]["mu"])
    stA = mlp.slots(pmA, 1, patA)
    nA = np.hypot(stA["a"], stA["b"])
    T = _first_update_transfer(stA["a"] / nA, stA["b"] / nA, lam0, mu0)      # [n, 3, 3]
    phi = mlp.basis(stA["a"], stA["b"])                                      # [27, n]
    C, *_ = np.linalg.lstsq(phi.T, T.reshape(-1, 9), rcond=None)             # [27, 9]
    o = C.T.ravel()                                                           # [(c 3 + d) 27 + n]
    pmB = random_discs(32, (2.0, 6.0), 0.4, seed=7)
    patB = O.pattern_adapted(pmB, 1, 150)
    macro = np.array([0.004, -0.007, 0, 0, 0, 0.003])
    r = O.solve(pmB, ph, macro, patB, tol=0.0, max_iter=1, scheme="continuous")
    _, null = wave_vector(np.asarray(patB), (32, 32, 1), "continuous")
    stB = mlp.slots(pmB, 1, patB, null)
    e, en = mlp.unit_direction(macro)
    p = mlp.head(o, stB, e)
    want = mlp.targets(r.eps_hat, pmB.size, macro, stB)
    assert np.allclose(p, want, rtol=1e-9, atol=1e-12 * np.abs(want).max())
    # conjugate frequencies get conjugate predictions (T is real and even)
    pat = np.asarray(patB)
    pos = {(int(kx), int(ky)): i for i, (kx, ky, _) in enumerate(pat[stB["index"]])}
    for i, (kx, ky, _) in enumerate(pat[stB["index"]]):
        j = pos.get((-int(kx), -int(ky)))
        if j is not None:
            assert np.allclose(p[j], np.conj(p[i]))


def test_head_one_hot_and_linearity():
    pm = random_discs(16, (2.0, 4.0), 0.3, seed=3)
    st = mlp.slots(pm, 1, O.pattern_adapted(pm, 1, 30))
    phi = mlp.basis(st["a"], st["b"])
    e = np.array([0.3, -0.5, 0.8])
    for c in range(3):
        for d in range(3):
            for n in (0, 5, 13, 26):
                o = np.zeros(mlp.N_OUT)
                o[(c * 3 + d) * mlp.N_BASIS + n] = 1.0
                p = mlp.head(o, st, e)
                want = np.zeros_like(p)
                want[:, c] = phi[n] * st["g"] * e[d]
                assert np.allclose(p, want)
    o = np.random.default_rng(1).standard_normal(mlp.N_OUT)
    assert np.allclose(mlp.head(o, st, 2 * e - e[::-1]),
                       2 * mlp.head(o, st, e) - mlp.head(o, st, e[::-1]))


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    hid, B = 6, 3
    shapes = [(mlp.N_DESC, hid), (hid,), (hid, hid), (hid,), (hid, mlp.N_OUT), (mlp.N_OUT,)]
    params = [rng.standard_normal(s) * 0.3 for s in shapes]
    X = rng.standard_normal((B, mlp.N_DESC))
    tables, targets = [], []
    for r in range(B):
        n = [5, 0, 9][r]                      # an RVE with no slots contributes nothing
        tables.append(dict(g=rng.standard_normal(n) + 1j * rng.standard_normal(n),
                           a=rng.uniform(-0.5, 0.5, n), b=rng.uniform(0.01, 0.5, n),
                           index=np.arange(n)))
        targets.append(rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3)))
    E = rng.standard_normal((B, 3))
    loss, grads = mlp.loss_and_grads(params, X, tables, targets, E)
    h = 1e-6
    for p, g in zip(params, grads):
        for idx in [tuple(rng.integers(0, n) for n in p.shape) for _ in range(5)]:
            old = p[idx]
            p[idx] = old + h
            lp, _ = mlp.loss_and_grads(params, X, tables, targets, E)
            p[idx] = old - h
            lm, _ = mlp.loss_and_grads(params, X, tables, targets, E)
            p[idx] = old
            assert math.isclose(g[idx], (lp - lm) / (2 * h), rel_tol=1e-6, abs_tol=1e-10)


def test_adam_first_step():
    p = [np.array([1.0, -2.0])]
    g = [np.array([0.5, -4.0])]
    st = ([np.zeros(2)], [np.zeros(2)], 0)
    newp, (m, v, t) = mlp.adam(p, g, st, lr=0.1)
    # first bias-corrected step moves every parameter by lr * g / (|g| + eps) ~ lr * sign(g)
    assert t == 1 and np.allclose(newp[0], [0.9, -1.9], atol=1e-7)
    assert np.allclose(m[0], 0.1 * g[0]) and np.allclose(v[0], 0.001 * g[0] ** 2)


def _full_pattern(n):
    return np.array([[kx, ky, 0] for ky in range(-(n - 1) // 2, n // 2 + 1)
                     for kx in range(-(n - 1) // 2, n // 2 + 1)])


def test_descriptors_sum_rules_and_symmetry():
    pm = centred_disc(24, 0.3)
    pat = _full_pattern(24)
    x = mlp.descriptors(pm, 1, pat)
    assert np.isclose(x[0], pm.mean())
    # Parseval: all nonzero power = vf - vf^2 (g^2 = g), split over the radial bins
    assert np.isclose(x[41] ** 2, pm.mean() - pm.mean() ** 2)
    assert np.isclose(np.sum(x[1:25] ** 2), x[41] ** 2)
    # a centred pixel disc is symmetric under 90-degree rotation and mirrors: no cos 2t, sin 2t
    assert np.allclose(x[25:41:4], 0, atol=1e-12) and np.allclose(x[26:41:4], 0, atol=1e-12)
    assert np.all(x[42:] == 0)
    # a laminate along x has all its power at ky = 0 (t = 0): cos 2t = cos 4t = 1 in every band
    lam = laminate((24, 24), (14, 10))           # layers normal to x: power only at ky = 0
    xl = mlp.descriptors(lam, 1, pat)
    band = [xl[25 + 4 * j:29 + 4 * j] for j in range(4) if xl[1 + 6 * j:7 + 6 * j].any()]
    assert band
    for c2, s2, c4, s4 in band:
        assert np.isclose(c2, 1.0) and np.isclose(s2, 0.0, atol=1e-12)
        assert np.isclose(c4, 1.0) and np.isclose(s4, 0.0, atol=1e-12)


def test_targets_pick_the_slot_components():
    rng = np.random.default_rng(3)
    pm = random_discs(16, (2.0, 4.0), 0.3, seed=5)
    pat = O.pattern_adapted(pm, 1, 20)
    st = mlp.slots(pm, 1, pat)
    K = len(pat)
    eh = rng.standard_normal((K, 3, 3)) + 1j * rng.standard_normal((K, 3, 3))
    eh = 0.5 * (eh + eh.transpose(0, 2, 1))
    macro = np.array([0.01, -0.004, 0, 0, 0, 0.003])
    t = mlp.targets(eh, pm.size, macro, st)
    _, en = mlp.unit_direction(macro)
    i = st["index"]
    assert np.allclose(t[:, 2], eh[i, 0, 1] / (pm.size * en))
    assert len(i) == K - 1 and not np.any(np.all(np.asarray(pat)[i, :2] == 0, axis=1))


def test_elastic_fixed_point_is_linear_in_macro_strain():
    """The head assumes linearity in ebar: every update of the scheme with linear phases is linear
    in (eps, ebar), so after the same number of updates the coefficients superpose exactly."""
    pm = centred_disc(16, 0.3)
    pat = O.pattern_adapted(pm, 1, 40)
    ph = elastic_phases()
    e1 = np.array([0.01, 0, 0, 0, 0, 0])
    e2 = np.array([0, 0.004, 0, 0, 0, -0.002])
    r1 = O.solve(pm, ph, e1, pat, tol=0.0, max_iter=6)
    r2 = O.solve(pm, ph, e2, pat, tol=0.0, max_iter=6)
    r12 = O.solve(pm, ph, 2 * e1 - 3 * e2, pat, tol=0.0, max_iter=6)
    assert np.allclose(r12.eps_hat, 2 * r1.eps_hat - 3 * r2.eps_hat, rtol=1e-10, atol=1e-12)
