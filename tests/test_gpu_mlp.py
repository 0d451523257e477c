"""Warm-start network kernels against the FP64 oracle (oracle/mlp.py), the batch hooks against
the solver's own outputs, and what the trained network gains over the plain start.

Tolerances: tensor-core operands are rounded to nearest, TF32 with unit roundoff u = 2^-11,
BF16 with u = 2^-9; a product of two rounded operands carries <= 2u relative error and sums
of random-signed products keep that order in the relative L2 norm. Three layers forward and
the chain rule backward compound a few such steps, so the relative L2 errors stay near
6u-10u: TF32 <= 1e-2 (forward 4e-3), BF16 <= 3e-2.
"""

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from oracle.rf_oracle import VOIGT
from synth import random_discs, random_macro_strain
from synth.configs import elastic_phases, k_target

pytestmark = pytest.mark.gpu

TF32_FWD, TF32_GRAD, BF16_FWD = 4e-3, 1e-2, 3e-2


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_net(lib, S=37, H=80, maxB=300, seed=1):
    net = lib.WarmStartNet(S, H, maxB)
    rng = np.random.default_rng(seed)
    parts = []
    for sh in net.shapes():
        fan = sh[0] if len(sh) == 2 else 4.0
        parts.append(rng.standard_normal(sh) / np.sqrt(fan))
    flat = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
    net.rf_mlp_set_params(flat)
    return net, [p.astype(np.float32).astype(np.float64) for p in net.split(flat)]


def test_forward_matches_oracle(lib):
    import torch
    net, params = make_net(lib)
    B = 300                                # three row tiles, the last one ragged
    rng = np.random.default_rng(2)
    X = rng.standard_normal((B, net.dims["n_in"])).astype(np.float32)
    want, _ = M.forward(params, X.astype(np.float64))
    dx = torch.as_tensor(X, device="cuda")
    for prec, tol in (("tf32", TF32_FWD), ("bf16", BF16_FWD)):
        got = net.rf_mlp_forward(dx, prec).cpu().numpy()
        assert got.shape == want.shape
        assert rel(got, want) <= tol, (prec, rel(got, want))
    net.close()


def test_gradients_match_oracle(lib):
    import torch
    net, params = make_net(lib, S=21, H=48, maxB=200, seed=3)
    S, B = 21, 200
    rng = np.random.default_rng(4)
    X = rng.standard_normal((B, 4 * S)).astype(np.float32)
    T = (0.3 * rng.standard_normal((B, 6 * S))).astype(np.float32)
    E = rng.standard_normal((B, 3))
    E = (E / np.linalg.norm(E, axis=1, keepdims=True)).astype(np.float32)
    valid = rng.integers(0, S + 1, B).astype(np.int32)
    valid[:5] = S
    mask = (np.arange(S)[None, :] < valid[:, None]).repeat(6, axis=1).astype(float)
    loss_o, grads_o = M.loss_and_grads(params, X.astype(np.float64), T.astype(np.float64),
                                       E.astype(np.float64), mask)
    d = [torch.as_tensor(a, device="cuda") for a in (X, T, E, valid)]
    loss = net.rf_mlp_loss_grad(*d)
    g = net.split(net.rf_mlp_get_grads())
    assert abs(loss - loss_o) <= TF32_GRAD * loss_o
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    for name, a, b in zip(names, g, grads_o):
        assert rel(a, b) <= TF32_GRAD, (name, rel(a, b))
    net.close()


def test_adam_step_matches_oracle(lib):
    import torch
    net, params = make_net(lib, S=9, H=32, maxB=64, seed=5)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((64, 36)).astype(np.float32)
    T = rng.standard_normal((64, 54)).astype(np.float32)
    E = np.tile(np.array([[0.6, 0.0, 0.8]], np.float32), (64, 1))
    valid = np.full(64, 9, np.int32)
    d = [torch.as_tensor(a, device="cuda") for a in (X, T, E, valid)]
    p0 = net.split(net.rf_mlp_get_params())
    state = ([np.zeros_like(p, dtype=np.float64) for p in p0],
             [np.zeros_like(p, dtype=np.float64) for p in p0], 0)
    p = [q.astype(np.float64) for q in p0]
    for lr in (1e-2, 5e-3, 2e-3):
        net.rf_mlp_loss_grad(*d, want_loss=False)
        g = [q.astype(np.float64) for q in net.split(net.rf_mlp_get_grads())]
        net.rf_mlp_adam(lr)
        p, state = M.adam(p, g, state, lr)      # the oracle's step on the kernel's gradients
        got = net.split(net.rf_mlp_get_params())
        for a, b in zip(got, p):
            assert np.allclose(a, b, rtol=1e-5, atol=1e-6)
        p = [q.astype(np.float64) for q in got]
    assert net.rf_mlp_get_dims()["adam_steps"] == 3
    net.close()


def population(n, side=24, seed0=700):
    pms, macros = [], []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        vf = float(rng.uniform(0.2, 0.5))
        pms.append(random_discs(side, (2.0, 5.0), vf, seed=seed0 + i))
        macros.append(random_macro_strain(seed0 + 5000 + i, 2))
    return pms, np.array(macros)


def test_batch_features_and_coefficients_match_oracle(lib):
    import torch
    pms, macros = population(5)
    pms[3] = np.ascontiguousarray(pms[3][:15])           # a rectangular (odd) cell
    pms[4] = random_discs(32, (2.0, 6.0), 0.35, seed=9)
    pats = [O.pattern_adapted(pm, 1, k_target(0.08, pm.size)) for pm in pms]
    S = max(len(p) for p in pats) - 3                    # some RVEs have fewer than S entries
    ph = elastic_phases()
    b = lib.BatchSolver(pms, ph, pats, tol=0.0, max_iter=6)
    out = b.rf_batch_solve(macros)
    assert np.all(out["iters"] == 6)
    x, v = b.rf_batch_features(S)
    c = b.rf_batch_reduced_strain(S).cpu().numpy()
    x = x.cpu().numpy()
    v = v.cpu().numpy()
    b.close()
    for i, (pm, pat) in enumerate(zip(pms, pats)):
        assert v[i] == min(S, len(pat))
        fo = M.features(pm, 1, pat, S)
        assert np.abs(x[i] - fo).max() <= 2e-6, i
        r = O.solve(pm, ph, macros[i], pat, tol=0.0, max_iter=6)
        want = np.zeros((S, 6, 2))
        for a, (p, q) in enumerate(VOIGT):
            n = min(S, len(pat))
            want[:n, a, 0] = r.eps_hat[:n, p, q].real
            want[:n, a, 1] = r.eps_hat[:n, p, q].imag
        assert rel(c[i], want) <= 1e-5, (i, rel(c[i], want))
        assert np.all(c[i, len(pat):] == 0)
    # targets from the exported coefficients
    net = lib.WarmStartNet(S, 16, 8)
    t, e = net.rf_mlp_targets(torch.as_tensor(c, device="cuda"),
                              torch.as_tensor(macros, dtype=torch.float64, device="cuda"),
                              torch.as_tensor([float(pm.size) for pm in pms],
                                              dtype=torch.float64, device="cuda"))
    t, e = t.cpu().numpy(), e.cpu().numpy()
    for i, pm in enumerate(pms):
        eh = np.zeros((S, 3, 3), complex)
        eh[:, 0, 0] = c[i, :, 0, 0] + 1j * c[i, :, 0, 1]
        eh[:, 1, 1] = c[i, :, 1, 0] + 1j * c[i, :, 1, 1]
        eh[:, 0, 1] = c[i, :, 5, 0] + 1j * c[i, :, 5, 1]
        assert np.allclose(t[i], M.targets(eh, pm.size, macros[i], S), rtol=1e-5, atol=1e-7)
        assert np.allclose(e[i], M.unit_direction(macros[i])[0], rtol=1e-6)
    net.close()


def test_device_warm_start_equals_host_warm_start(lib):
    import torch
    pms, macros = population(4, seed0=800)
    pats = [O.pattern_adapted(pm, 1, k_target(0.08, pm.size)) for pm in pms]
    ph = elastic_phases()
    S = max(len(p) for p in pats)
    host, dev = [], np.zeros((len(pms), S, 6, 2), np.float32)
    for i, (pm, pat) in enumerate(zip(pms, pats)):
        r = O.solve(pm, ph, macros[i], pat, tol=1e-9, max_iter=3000)
        w = np.zeros((len(pat), 6, 2), np.float32)
        for a, (p, q) in enumerate(VOIGT):
            w[:, a, 0] = r.eps_hat[:, p, q].real
            w[:, a, 1] = r.eps_hat[:, p, q].imag
        host.append(w)
        dev[i, :len(pat)] = w
    b = lib.BatchSolver(pms, ph, pats, tol=1e-6, max_iter=2000)
    a = b.rf_batch_solve(macros, warm=host)
    d = b.rf_batch_solve_warm(macros, torch.as_tensor(dev, device="cuda"), S)
    b.close()
    assert np.array_equal(a["iters"], d["iters"]) and np.all(d["iters"] <= 2)
    assert np.array_equal(a["sigma_bar"], d["sigma_bar"])
