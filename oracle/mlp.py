"""FP64 CPU oracle of the warm-start network (test infrastructure only).

Written from the definitions below with numpy; every gradient is pinned by central finite
differences and the head by the scheme's first update (tests/test_oracle_mlp.py).

One 2D RVE: grid (Ny, Nx), N voxels, inclusion indicator g, pattern list of K frequencies
k = (kx, ky) (Sec. 4). gamma(k) = g^(k) / N with g^(k) = sum_x g(x) exp(-2 pi i (kx x / Nx +
ky y / Ny)); a = kx / Nx, b = ky / Ny (cycles per voxel), rho = sqrt(a^2 + b^2).

Descriptors x [48] of the RVE (the network input):
  x[0]       volume fraction gamma(0)
  x[1 + i]   sqrt(sum |gamma|^2) over the nonzero pattern frequencies with radial bin i,
             i = min(23, floor(96 rho)) (24 bins of width 1/96; the bin is decided in FP64)
  x[25 + 4 j + m]  sum |gamma|^2 h_m / (sum |gamma|^2 + 1e-12) over radial band j = i // 6
             (4 bands), h = (cos 2t, sin 2t, cos 4t, sin 4t), t the angle of (a, b)
  x[41]      sqrt(sum |gamma|^2) over all nonzero pattern frequencies; x[42:48] = 0
Network: h1 = GELU(x W1 + b1), h2 = GELU(h1 W2 + b2), o = h2 W3 + b3 (48 -> H -> H -> 243),
GELU(z) = z Phi(z) with the standard normal CDF Phi.
Head: o holds a real strain-transfer expansion C[c 3 + d][n] = o[(c 3 + d) 27 + n] over 27 basis
functions phi_n(a, b) = r_i(rho) h_j(t), n = 9 i + j, r = (1, rho / 0.25, (rho / 0.25)^2),
h = (1, cos 2t, sin 2t, cos 4t, sin 4t, cos 6t, sin 6t, cos 8t, sin 8t); the harmonics are the
rational functions of (a, b) (cos 2t = (a^2 - b^2) / rho^2, sin 2t = 2 a b / rho^2, and the
double- and sum-angle formulas). For a nonzero, non-null pattern frequency the prediction is
  p_c(k) = sum_d T_cd(k) gamma(k) e_d,   T_cd(k) = sum_n C[c 3 + d][n] phi_n(k),
c, d over strain components (11, 22, 12), e = (ebar_11, ebar_22, ebar_12) / |ebar| (Frobenius).
T is real and even in k, so p(-k) = conj(p(k)) as for a real field, and p is linear in ebar and
in gamma: the structure of the scheme's first update (Sec. 4, step c applied to the plain start).
Targets: t_c(k) = eps^_c(k) / (N |ebar|) of the converged reduced solution.
Loss: mean of (Re, Im of p - t)^2 over the slots (all nonzero non-null pattern frequencies of
the batch, 6 reals each), minimised with Adam.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

N_DESC = 48
N_BASIS = 27
N_OUT = 9 * N_BASIS
N_BINS = 24
BIN_SCALE = 96.0
RHO_REF = 0.25


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def harmonics(a, b):
    """(1, cos 2t, sin 2t, cos 4t, sin 4t, cos 6t, sin 6t, cos 8t, sin 8t) of the angle t of
    (a, b) != 0, from the rational forms; shape [9, n]."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    r2 = a * a + b * b
    c2, s2 = (a * a - b * b) / r2, 2.0 * a * b / r2
    c4, s4 = c2 * c2 - s2 * s2, 2.0 * s2 * c2
    c6, s6 = c4 * c2 - s4 * s2, s4 * c2 + c4 * s2
    c8, s8 = c4 * c4 - s4 * s4, 2.0 * s4 * c4
    return np.array([np.ones_like(a), c2, s2, c4, s4, c6, s6, c8, s8])


def basis(a, b):
    """phi [27, n]: radial (1, rho~, rho~^2) x harmonics, n = 9 i + j."""
    rho = np.sqrt(np.asarray(a, float) ** 2 + np.asarray(b, float) ** 2) / RHO_REF
    h = harmonics(a, b)
    return np.concatenate([h, h * rho, h * rho * rho])


def _gamma(phase_map, inclusion_phase, pattern):
    pm = np.asarray(phase_map)
    ny, nx = pm.shape
    g = (pm == inclusion_phase).astype(float)
    G = np.fft.fft2(g) / pm.size
    pat = np.asarray(pattern)
    return np.array([G[ky % ny, kx % nx] for kx, ky, _ in pat]), nx, ny


def slots(phase_map, inclusion_phase, pattern, null=None):
    """Slot table of one RVE: the nonzero, non-null pattern entries (pattern order) with
    gamma, a, b and their pattern indices. `null` [K] marks the frequencies the Green operator
    sets to zero (Sec. 4 step c)."""
    gam, nx, ny = _gamma(phase_map, inclusion_phase, pattern)
    pat = np.asarray(pattern)
    keep = ~np.all(pat[:, :2] == 0, axis=1)
    if null is not None:
        keep &= ~np.asarray(null, bool)
    idx = np.nonzero(keep)[0]
    return dict(g=gam[idx], a=pat[idx, 0] / nx, b=pat[idx, 1] / ny, index=idx)


def descriptors(phase_map, inclusion_phase, pattern):
    gam, nx, ny = _gamma(phase_map, inclusion_phase, pattern)
    pat = np.asarray(pattern)
    x = np.zeros(N_DESC)
    nz = ~np.all(pat[:, :2] == 0, axis=1)
    x[0] = gam[~nz][0].real
    a = pat[nz, 0] / nx
    b = pat[nz, 1] / ny
    p = np.abs(gam[nz]) ** 2
    bins = np.minimum(N_BINS - 1, np.floor(BIN_SCALE * np.sqrt(a * a + b * b)).astype(int))
    h = harmonics(a, b)
    for i in range(N_BINS):
        x[1 + i] = math.sqrt(p[bins == i].sum())
    for j in range(4):
        sel = bins // 6 == j
        tot = p[sel].sum()
        for m in range(4):
            x[25 + 4 * j + m] = (p[sel] * h[1 + m][sel]).sum() / (tot + 1e-12)
    x[41] = math.sqrt(p.sum())
    return x


def unit_direction(macro):
    """e^ = (ebar_11, ebar_22, ebar_12) / |ebar|_F and |ebar|_F (Voigt order 11 22 33 23 13 12)."""
    e = np.asarray(macro, float)
    en = math.sqrt(e[0] ** 2 + e[1] ** 2 + e[2] ** 2 + 2 * (e[3] ** 2 + e[4] ** 2 + e[5] ** 2))
    return np.array([e[0], e[1], e[5]]) / en, en


def targets(eps_hat, N, macro, slot_table):
    """t [n, 3] complex: eps^_c / (N |ebar|) at the slots; eps_hat [K, 3, 3] in pattern order."""
    _, en = unit_direction(macro)
    eh = np.asarray(eps_hat)[slot_table["index"]]
    return np.stack([eh[:, 0, 0], eh[:, 1, 1], eh[:, 0, 1]], axis=1) / (N * en)


def forward(params, X):
    """params = (W1, b1, W2, b2, W3, b3), W_l of shape [in, out]. Returns (out, cache)."""
    W1, b1, W2, b2, W3, b3 = params
    Z1 = X @ W1 + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2 + b2
    H2 = gelu(Z2)
    O = H2 @ W3 + b3
    return O, (X, Z1, H1, Z2, H2)


def transfer(o, slot_table):
    """T [n, 3, 3] (c, d) from one RVE's output o [243]."""
    C = np.asarray(o).reshape(9, N_BASIS)
    phi = basis(slot_table["a"], slot_table["b"])
    return (C @ phi).T.reshape(-1, 3, 3)


def head(o, slot_table, ehat):
    """p [n, 3] complex for one RVE."""
    T = transfer(o, slot_table)
    return np.einsum("scd,d->sc", T, ehat) * slot_table["g"][:, None]


def loss_and_grads(params, X, slot_tables, T_list, E):
    """Loss over a batch of RVEs (X [B, 48], slot tables, targets [n_b, 3] complex, unit
    directions E [B, 3]) and its gradients with respect to every parameter."""
    W1, b1, W2, b2, W3, b3 = params
    O, (X, Z1, H1, Z2, H2) = forward(params, X)
    count = 6.0 * sum(len(st["g"]) for st in slot_tables)
    loss = 0.0
    dO = np.zeros_like(O)
    for r, (st, t) in enumerate(zip(slot_tables, T_list)):
        if len(st["g"]) == 0:
            continue
        p = head(O[r], st, E[r])
        res = p - t
        loss += float(np.sum(res.real ** 2 + res.imag ** 2))
        # dL/dT_cd(s) = 2 / count * Re(conj(res_c) g) e_d ; dC = sum_s dT(s) phi(s)
        w = 2.0 / count * (np.conj(res) * st["g"][:, None]).real          # [n, 3]
        dT = w[:, :, None] * E[r][None, None, :]                           # [n, 3, 3]
        phi = basis(st["a"], st["b"])                                      # [27, n]
        dO[r] = (dT.reshape(-1, 9).T @ phi.T).ravel()
    loss /= count
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


def warm_coefficients(o, slot_table, N, macro, K):
    """Starting coefficients [K, 3, 3] complex (pattern order) from one RVE's output o: N |ebar|
    times the prediction at the slots, zero elsewhere (the solver sets the zero frequency)."""
    e, en = unit_direction(macro)
    p = head(o, slot_table, e) * (N * en)
    w = np.zeros((K, 3, 3), complex)
    idx = slot_table["index"]
    w[idx, 0, 0] = p[:, 0]
    w[idx, 1, 1] = p[:, 1]
    w[idx, 0, 1] = w[idx, 1, 0] = p[:, 2]
    return w
