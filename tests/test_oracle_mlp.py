"""Pins of the warm-start network oracle: GELU against its closed form and values, gradients
against central finite differences, the head's index layout against one-hot outputs, Adam against
a hand-worked first step, features against the DFT definition and the zero frequency's volume
fraction, and the premise of the head (the elastic fixed point is linear in ebar) against the
scheme itself."""

import math

import numpy as np

import oracle as O
from oracle import mlp
from synth import centred_disc
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


def test_head_layout_one_hot():
    S = 3
    ehat = np.array([[0.2, -0.5, 0.7]])
    for s in range(S):
        for c in range(3):
            for d in range(3):
                for r in range(2):
                    Oo = np.zeros((1, 18 * S))
                    Oo[0, ((s * 3 + c) * 3 + d) * 2 + r] = 1.0
                    P = mlp.head(Oo, ehat)
                    want = np.zeros((1, 6 * S))
                    want[0, (s * 3 + c) * 2 + r] = ehat[0, d]
                    assert np.array_equal(P, want)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    S, hid, B = 2, 6, 3
    shapes = [(4 * S, hid), (hid,), (hid, hid), (hid,), (hid, 18 * S), (18 * S,)]
    params = [rng.standard_normal(s) * 0.5 for s in shapes]
    X = rng.standard_normal((B, 4 * S))
    T = rng.standard_normal((B, 6 * S))
    ehat = rng.standard_normal((B, 3))
    mask = np.ones((B, 6 * S))
    mask[1, 6:] = 0.0          # sample 1 has one valid slot
    loss, grads = mlp.loss_and_grads(params, X, T, ehat, mask)
    h = 1e-6
    for p, g in zip(params, grads):
        for idx in [tuple(rng.integers(0, n) for n in p.shape) for _ in range(5)]:
            old = p[idx]
            p[idx] = old + h
            lp, _ = mlp.loss_and_grads(params, X, T, ehat, mask)
            p[idx] = old - h
            lm, _ = mlp.loss_and_grads(params, X, T, ehat, mask)
            p[idx] = old
            assert math.isclose(g[idx], (lp - lm) / (2 * h), rel_tol=1e-6, abs_tol=1e-9)
    # output units of slot 1 get gradient only from the samples where slot 1 is valid
    X1 = X.copy()
    mask_only1 = np.zeros_like(mask)
    mask_only1[1] = mask[1]
    _, g1 = mlp.loss_and_grads(params, X1, T, ehat, mask_only1)
    assert np.all(g1[5][18:] == 0)


def test_adam_first_step():
    p = [np.array([1.0, -2.0])]
    g = [np.array([0.5, -4.0])]
    st = ([np.zeros(2)], [np.zeros(2)], 0)
    newp, (m, v, t) = mlp.adam(p, g, st, lr=0.1)
    # first bias-corrected step moves every parameter by lr * g / (|g| + eps) ~ lr * sign(g)
    assert t == 1 and np.allclose(newp[0], [0.9, -1.9], atol=1e-7)
    assert np.allclose(m[0], 0.1 * g[0]) and np.allclose(v[0], 0.001 * g[0] ** 2)


def test_features_match_definition():
    pm = centred_disc(12, 0.3)
    pat = np.array([[0, 0, 0], [1, 2, 0], [-1, -2, 0]])
    f = mlp.features(pm, 1, pat, 4)
    assert np.isclose(f[0], pm.mean()) and f[1] == 0.0      # g^(0)/N = volume fraction
    gh = np.fft.fft2((pm == 1).astype(float))[2, 1] / pm.size
    assert np.isclose(f[4], gh.real) and np.isclose(f[5], gh.imag)
    assert np.allclose(f[6:8], [1 / 12, 2 / 12])
    assert np.isclose(f[8], gh.real) and np.isclose(f[9], -gh.imag)   # conjugate frequency
    assert np.all(f[12:16] == 0)                               # missing slot


def test_targets_and_warm_coefficients_round_trip():
    rng = np.random.default_rng(3)
    K, S, N = 7, 5, 144
    eh = rng.standard_normal((K, 3, 3)) + 1j * rng.standard_normal((K, 3, 3))
    eh = 0.5 * (eh + eh.transpose(0, 2, 1))
    macro = np.array([0.01, -0.004, 0, 0, 0, 0.003])
    t = mlp.targets(eh, N, macro, S)
    w = mlp.warm_coefficients(t, N, macro, K)
    for s in range(S):
        assert np.allclose(w[s, [0, 1, 5], 0], [eh[s, 0, 0].real, eh[s, 1, 1].real, eh[s, 0, 1].real])
        assert np.allclose(w[s, [0, 1, 5], 1], [eh[s, 0, 0].imag, eh[s, 1, 1].imag, eh[s, 0, 1].imag])
    assert np.all(w[S:] == 0) and np.all(w[:, 2:5] == 0)


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
    # so does the target scaled by 1/(N |ebar|), contracted with the unit direction
    t1 = mlp.targets(r1.eps_hat, pm.size, e1, 10)
    t1s = mlp.targets(O.solve(pm, ph, 5 * e1, pat, tol=0.0, max_iter=6).eps_hat, pm.size, 5 * e1, 10)
    assert np.allclose(t1, t1s, rtol=1e-10, atol=1e-14)
