"""FP64 CPU oracle of the warm-start network (test infrastructure only).

A three-layer perceptron, in -> hidden -> hidden -> out, with GELU activations
GELU(z) = z * Phi(z) = 0.5 z (1 + erf(z / sqrt 2)), a linear output head, mean-squared-error
loss over the valid outputs, and Adam updates. Written from these definitions with numpy; its
gradients are pinned by central finite differences (tests/test_oracle_mlp.py).

Inputs of one 2D RVE: the transform of the phase indicator g and the wave numbers at the first
n_slots frequencies of its pattern (pattern order). The network output holds, per slot, strain
component c in (11, 22, 12) and macroscopic-strain direction d in (11, 22, 12), a complex
strain-concentration coefficient A[s, c, d]; the head contracts it with the unit direction
e^ = (ebar_11, ebar_22, ebar_12) / |ebar| of the macroscopic strain, so the prediction is exactly
linear in ebar, as the elastic fixed point is (Sec. 4, the scheme is linear for linear phases).
Targets are the converged reduced strain coefficients scaled by 1 / (N |ebar|), |ebar| the
Frobenius norm.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, X):
    """params = (W1, b1, W2, b2, W3, b3), W_l of shape [in, out]. Returns (out, cache)."""
    W1, b1, W2, b2, W3, b3 = params
    Z1 = X @ W1 + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2 + b2
    H2 = gelu(Z2)
    O = H2 @ W3 + b3
    return O, (X, Z1, H1, Z2, H2)


def head(O, ehat):
    """P[b, (s, c, r)] = sum_d O[b, (s, c, d, r)] ehat[b, d]; O [B, 18 S], ehat [B, 3]."""
    B = O.shape[0]
    A = O.reshape(B, -1, 3, 3, 2)
    return np.einsum("bscdr,bd->bscr", A, ehat).reshape(B, -1)


def loss_and_grads(params, X, T, ehat, mask=None):
    """Mean squared error of the head's prediction over the valid entries (mask [B, 6 S] of 0/1)
    and its gradients with respect to every parameter."""
    W1, b1, W2, b2, W3, b3 = params
    O, (X, Z1, H1, Z2, H2) = forward(params, X)
    P = head(O, ehat)
    m = np.ones_like(P) if mask is None else np.asarray(mask, float)
    count = m.sum()
    R = (P - T) * m
    loss = float(np.sum(R * R) / count)
    dP = 2.0 * R / count
    B = O.shape[0]
    dO = np.einsum("bscr,bd->bscdr", dP.reshape(B, -1, 3, 2), ehat).reshape(B, -1)
    dW3 = H2.T @ dO
    db3 = dO.sum(0)
    dZ2 = (dO @ W3.T) * gelu_grad(Z2)
    dW2 = H1.T @ dZ2
    db2 = dZ2.sum(0)
    dZ1 = (dZ2 @ W2.T) * gelu_grad(Z1)
    dW1 = X.T @ dZ1
    db1 = dZ1.sum(0)
    return loss, (dW1, db1, dW2, db2, dW3, db3)


def adam(params, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected); state = (m, v, t). Returns new params and state."""
    m, v, t = state
    t += 1
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = b1 * mm + (1 - b1) * g
        vv = b2 * vv + (1 - b2) * g * g
        mh = mm / (1 - b1 ** t)
        vh = vv / (1 - b2 ** t)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, (out_m, out_v, t)


def unit_direction(macro):
    """e^ = (ebar_11, ebar_22, ebar_12) / |ebar|_F and |ebar|_F (Voigt order 11 22 33 23 13 12)."""
    e = np.asarray(macro, float)
    en = math.sqrt(e[0] ** 2 + e[1] ** 2 + e[2] ** 2 + 2 * (e[3] ** 2 + e[4] ** 2 + e[5] ** 2))
    return np.array([e[0], e[1], e[5]]) / en, en


def features(phase_map, inclusion_phase, pattern, n_slots):
    """Input vector of one 2D RVE: for slot s < n_slots (the s-th pattern frequency, pattern order)
    Re g^ / N, Im g^ / N, kx / Nx, ky / Ny, with g^(k) = sum_x g(x) exp(-2 pi i k.x / N_grid).
    Missing slots are zero."""
    pm = np.asarray(phase_map)
    ny, nx = pm.shape
    N = pm.size
    g = (pm == inclusion_phase).astype(float)
    y, x = np.mgrid[0:ny, 0:nx]
    f = np.zeros(4 * n_slots)
    for s, (kx, ky, _) in enumerate(np.asarray(pattern)[:n_slots]):
        gh = np.sum(g * np.exp(-2j * np.pi * (kx * x / nx + ky * y / ny))) / N
        f[4 * s:4 * s + 4] = (gh.real, gh.imag, kx / nx, ky / ny)
    return f


def targets(eps_hat, N, macro, n_slots):
    """Output vector: slot s holds Re, Im of eps^_11, eps^_22, eps^_12 scaled by 1 / (N |ebar|),
    |ebar| the Frobenius norm; eps_hat [K, 3, 3] in pattern order."""
    _, en = unit_direction(macro)
    t = np.zeros(6 * n_slots)
    for s in range(min(n_slots, len(eps_hat))):
        v = eps_hat[s]
        c = np.array([v[0, 0], v[1, 1], v[0, 1]]) / (N * en)
        t[6 * s:6 * s + 6] = (c[0].real, c[0].imag, c[1].real, c[1].imag, c[2].real, c[2].imag)
    return t


def warm_coefficients(P, N, macro, K):
    """Starting coefficients [K, 6, 2] (Voigt order, real/imaginary) from one prediction
    P [6 S]: slot s < min(S, K) gets N |ebar| P for 11, 22, 12; the rest are zero."""
    _, en = unit_direction(macro)
    S = P.size // 6
    w = np.zeros((K, 6, 2))
    for s in range(min(S, K)):
        for c, v in enumerate((0, 1, 5)):
            w[s, v, 0] = N * en * P[6 * s + 2 * c]
            w[s, v, 1] = N * en * P[6 * s + 2 * c + 1]
    return w
