"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test ties one oracle function to something other than itself: brute-force sums written
from the DFT definition, the closed-form isotropic Green operator and its projector identities,
closed-form solutions (homogeneous medium, empty reduced set = Voigt, laminate), variational
bounds (nested reduced sets, Hashin-Shtrikman), the J2 uniaxial-strain closed form, and a dense
brute-force solve of the reduced (Galerkin) system.
"""

import numpy as np
import pytest

import oracle as O
from oracle.rf_oracle import _as_grid
from synth import centred_disc, laminate, phase_table, random_discs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

TWO_PHASE = phase_table([(40.38, 26.92, 0.0, 0.0, 0), (111.1, 166.7, 0.0, 0.0, 0)])


def random_closed_pattern(shape_zyx, n_pick, seed):
    """Random reduced set: zero + n_pick random points + their conjugates."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    sidx = lambda i, n: i if i <= n // 2 else i - n  # noqa: E731
    pts = {(0, 0, 0)}
    for _ in range(n_pick):
        ix, iy, iz = rng.integers(nx), rng.integers(ny), rng.integers(nz)
        k = (sidx(ix, nx), sidx(iy, ny), sidx(iz, nz))
        c = (sidx((-k[0]) % nx, nx), sidx((-k[1]) % ny, ny), sidx((-k[2]) % nz, nz))
        pts.add(k)
        pts.add(c)
    return np.array(sorted(pts), np.int64)


def brute_forward(field, pattern):
    nz, ny, nx = field.shape[:3]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = []
    for kx, ky, kz in pattern:
        ph = np.exp(-2j * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz))
        out.append(np.tensordot(ph, field, axes=([0, 1, 2], [0, 1, 2])))
    return np.array(out)


def brute_inverse(coeffs, pattern, shape_zyx):
    nz, ny, nx = shape_zyx
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = 0
    for c, (kx, ky, kz) in zip(coeffs, pattern):
        ph = np.exp(2j * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz))
        f = f + ph[(...,) + (None,) * (np.ndim(c))] * c
    return np.real(f) / (nx * ny * nz)


# ----------------------------------------------------------------------------- transforms
@pytest.mark.parametrize("shape", [(1, 8, 8), (4, 4, 4), (1, 6, 10), (3, 5, 7)])
def test_transforms_match_bruteforce_dft(shape):
    rng = np.random.default_rng(1)
    field = rng.standard_normal(shape + (3, 3))
    pat = random_closed_pattern(shape, 9, 2)
    got = O.forward_reduced(field, pat)
    want = brute_forward(field, pat)
    assert np.allclose(got, want, atol=1e-11)
    back = O.inverse_reduced(want, pat, shape)
    assert np.allclose(back, brute_inverse(want, pat, shape), atol=1e-12)


def test_parseval_on_band_limited_field():
    shape = (1, 8, 12)
    pat = random_closed_pattern(shape, 15, 3)
    rng = np.random.default_rng(4)
    field = rng.standard_normal(shape)
    c = O.forward_reduced(field, pat)
    band = O.inverse_reduced(c, pat, shape)       # band-limited to the pattern
    cb = O.forward_reduced(band, pat)
    n = np.prod(shape)
    assert np.isclose(np.mean(band ** 2), np.sum(np.abs(cb) ** 2) / n ** 2, rtol=1e-12)


# ----------------------------------------------------------------------------- Green operator
def gamma_closed_form(q, lam0, mu0):
    d = np.eye(3)
    out = np.zeros((len(q), 3, 3, 3, 3))
    for m, v in enumerate(q):
        n2 = v @ v
        if n2 == 0:
            continue
        t1 = (np.einsum("ki,l,j->ijkl", d, v, v) + np.einsum("li,k,j->ijkl", d, v, v)
              + np.einsum("kj,l,i->ijkl", d, v, v) + np.einsum("lj,k,i->ijkl", d, v, v))
        t2 = np.einsum("i,j,k,l->ijkl", v, v, v, v)
        out[m] = t1 / (4 * mu0 * n2) - (lam0 + mu0) / (mu0 * (lam0 + 2 * mu0)) * t2 / n2 ** 2
    return out


def test_green_operator_closed_form_and_projector():
    rng = np.random.default_rng(5)
    q = rng.standard_normal((20, 3))
    q[3, 2] = 0.0
    lam0, mu0 = 3.7, 1.9
    G = O.green_operator(q, lam0, mu0)
    assert np.allclose(G, gamma_closed_form(q, lam0, mu0), atol=1e-13)
    C0 = O.isotropic_stiffness(lam0, mu0)
    for m in range(len(q)):
        g = G[m]
        assert np.allclose(g, g.transpose(1, 0, 2, 3)) and np.allclose(g, g.transpose(2, 3, 0, 1))
        P = np.einsum("ijab,abkl->ijkl", g, C0)
        assert np.allclose(np.einsum("ijab,abkl->ijkl", P, P), P, atol=1e-12)      # projector
        u = rng.standard_normal(3)
        s = 0.5 * (np.outer(q[m], u) + np.outer(u, q[m]))
        assert np.allclose(np.einsum("ijkl,kl->ij", P, s), s, atol=1e-12)           # compatible
    assert np.all(O.green_operator(np.zeros((1, 3)), lam0, mu0) == 0)


def test_wave_vector_rotated_and_continuous():
    pat = np.array([[0, 0, 0], [1, 0, 0], [4, 0, 0], [4, 4, 0], [2, -3, 0]])
    q, null = O.wave_vector(pat, (8, 8, 1), "rotated")
    t = np.pi * np.array([2, -3]) / 8
    assert np.allclose(q[4], [2 * np.sin(t[0]) * np.cos(t[1]), 2 * np.sin(t[1]) * np.cos(t[0]), 0])
    assert np.allclose(q[2], [2, 0, 0])                     # single Nyquist component
    assert list(null) == [False, False, False, True, False]  # two Nyquist components -> q = 0
    qc, nullc = O.wave_vector(pat, (8, 8, 1), "continuous")
    assert np.allclose(qc[1], [2 * np.pi / 8, 0, 0])
    assert list(nullc) == [False, False, True, True, False]


# ----------------------------------------------------------------------------- closed forms
def c_apply(lam, mu, e):
    return lam * np.trace(e) * np.eye(3) + 2 * mu * e


def test_homogeneous_medium_converges_in_one_step():
    pm = np.zeros((8, 8), np.uint8)
    pm[2:5, 3:7] = 1
    ph = phase_table([(2.0, 1.5, 0, 0, 0), (2.0, 1.5, 0, 0, 0)])
    pat = O.pattern_adapted(pm, 1, 13)
    ebar = np.array([0.01, -0.004, 0, 0, 0, 0.002])
    r = O.solve(pm, ph, ebar, pat, tol=1e-12)
    assert r.iters == 1 and r.residual == 0.0
    want = O.tensor_to_vec6(c_apply(2.0, 1.5, O.vec6_to_tensor(ebar)))
    assert np.allclose(r.sigma_bar, want, rtol=1e-14, atol=1e-16)


def test_zero_only_pattern_gives_voigt():
    pm = centred_disc(16, 0.3)
    ebar = np.array([0.01, 0.003, 0, 0, 0, -0.002])
    r = O.solve(pm, TWO_PHASE, ebar, np.zeros((1, 3), np.int64), tol=1e-12)
    f = pm.mean()
    E = O.vec6_to_tensor(ebar)
    want = (1 - f) * c_apply(TWO_PHASE["lam"][0], TWO_PHASE["mu"][0], E) \
        + f * c_apply(TWO_PHASE["lam"][1], TWO_PHASE["mu"][1], E)
    assert np.allclose(r.sigma_bar, O.tensor_to_vec6(want), rtol=1e-13)
    assert np.allclose(r.eps, E)


def laminate_closed_form(lams, mus, fracs, ebar):
    """Layers normal to x, plane strain: sigma_11, sigma_12 uniform; eps_22 = ebar_22."""
    lams, mus, fr = map(np.asarray, (lams, mus, fracs))
    e11, e22, e12 = ebar[0], ebar[1], ebar[5]
    s11 = (e11 + e22 * np.sum(fr * lams / (lams + 2 * mus))) / np.sum(fr / (lams + 2 * mus))
    s12 = e12 / np.sum(fr / (2 * mus))
    eps11 = (s11 - lams * e22) / (lams + 2 * mus)
    s22 = lams * (eps11 + e22) + 2 * mus * e22
    s33 = lams * (eps11 + e22)
    return s11, s12, eps11, s22, s33


@pytest.mark.parametrize("reduced", [False, True])
def test_laminate_closed_form(reduced):
    pm = laminate((6, 16), (5, 11))
    ebar = np.array([0.01, -0.004, 0, 0, 0, 0.003])
    if reduced:
        pat = O.pattern_adapted(pm, 1, 16)
        assert np.all(pat[:, 1] == 0) and len(pat) == 16     # the whole k_y = 0 axis
    else:
        pat = O.pattern_adapted(pm, 1, pm.size)
    r = O.solve(pm, TWO_PHASE, ebar, pat, tol=1e-13, max_iter=5000)
    s11, s12, e11, s22, s33 = laminate_closed_form(TWO_PHASE["lam"], TWO_PHASE["mu"],
                                                   (5 / 16, 11 / 16), ebar)
    sig = r.sigma[0]
    ph = pm.astype(int)
    assert np.allclose(sig[..., 0, 0], s11, rtol=1e-10)
    assert np.allclose(sig[..., 0, 1], s12, rtol=1e-10)
    assert np.allclose(r.eps[0][..., 0, 0], e11[ph], rtol=1e-10)
    assert np.allclose(r.eps[0][..., 1, 1], ebar[1], rtol=1e-10)
    assert np.allclose(sig[..., 1, 1], s22[ph], rtol=1e-10)
    assert np.allclose(sig[..., 2, 2], s33[ph], rtol=1e-10)


def test_nested_reduced_sets_energy_is_monotone():
    pm = centred_disc(16, 0.3)
    ebar = np.array([0.01, -0.003, 0, 0, 0, 0.004])
    E = O.vec6_to_tensor(ebar)
    energies, prev = [], None
    for K in (1, 9, 21, 41, 81, 161, 256):
        pat = O.pattern_adapted(pm, 1, K)
        s = {tuple(p) for p in pat}
        if prev is not None:
            assert prev <= s                      # nested: a prefix of one order
        prev = s
        r = O.solve(pm, TWO_PHASE, ebar, pat, tol=1e-12, max_iter=5000)
        energies.append(np.sum(O.vec6_to_tensor(r.sigma_bar) * E))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(energies, energies[1:]))
    assert energies[0] > energies[-1]


def test_bulk_modulus_inside_hashin_shtrikman_bounds():
    pm = random_discs(32, (4.0, 7.0), 0.35, seed=7)
    f = pm.mean()
    e = 0.01
    ebar = np.array([e, e, 0, 0, 0, 0])
    lam, mu = TWO_PHASE["lam"], TWO_PHASE["mu"]
    km, kf = lam[0] + mu[0], lam[1] + mu[1]
    lo = km + f / (1 / (kf - km) + (1 - f) / (km + mu[0]))
    hi = kf + (1 - f) / (1 / (km - kf) + f / (kf + mu[1]))
    for K in (pm.size, O_k(pm, 0.05)):
        pat = O.pattern_adapted(pm, 1, K)
        r = O.solve(pm, TWO_PHASE, ebar, pat, tol=1e-10, max_iter=5000)
        kstar = (r.sigma_bar[0] + r.sigma_bar[1]) / (2 * 2 * e)
        assert lo <= kstar <= hi, (lo, kstar, hi)


def O_k(pm, ratio):
    return int(np.ceil(ratio * pm.size - 1e-9))


# ----------------------------------------------------------------------------- J2
def j2_uniaxial(e, lam, mu, sy, H):
    kappa = lam + 2 * mu / 3
    if 2 * mu * abs(e) <= sy:
        alpha, seq = 0.0, 2 * mu * e
    else:
        alpha = (2 * mu * e - sy) / (3 * mu + H)
        seq = 2 * mu * e - 3 * mu * alpha
    return kappa * e + 2 / 3 * seq, kappa * e - seq / 3, alpha


def test_j2_return_map_uniaxial_strain_closed_form():
    lam, mu, sy, H = 40.4, 26.9, 0.25, 1.0
    for e in np.linspace(0.0, 0.03, 13):
        eps = np.zeros((1, 3, 3))
        eps[0, 0, 0] = e
        s, ep, a, _ = O.law(eps, [lam], [mu], [sy], [H], [True])
        s11, s22, alpha = j2_uniaxial(e, lam, mu, sy, H)
        assert np.isclose(s[0, 0, 0], s11, rtol=1e-13, atol=1e-15)
        assert np.isclose(s[0, 1, 1], s22, rtol=1e-13, atol=1e-15)
        assert np.isclose(s[0, 2, 2], s22, rtol=1e-13, atol=1e-15)
        assert np.isclose(a[0], alpha, rtol=1e-13, atol=1e-16)
        assert abs(np.trace(ep[0])) < 1e-16                        # plastic flow is deviatoric


def test_homogeneous_j2_path_one_step_per_increment():
    pm = np.zeros((4, 6), np.uint8)
    ph = phase_table([(40.4, 26.9, 0.25, 1.0, 1)])
    path = np.zeros((10, 6))
    path[:, 0] = np.linspace(0.002, 0.02, 10)
    pat = O.pattern_adapted(pm, 1, 5)
    sbar, iters, _ = O.solve_path(pm, ph, path, pat, tol=1e-10)
    assert np.all(iters == 1)
    for n in range(10):
        s11, s22, _ = j2_uniaxial(path[n, 0], 40.4, 26.9, 0.25, 1.0)
        assert np.isclose(sbar[n, 0], s11, rtol=1e-12) and np.isclose(sbar[n, 1], s22, rtol=1e-12)


def test_homogeneous_j2_load_unload_reload_closed_form():
    """Uniaxial strain eps_11 up to 2 %, back to 1.6 %, then on to 2.5 % (Sec. 2: yield
    function, associative flow, linear isotropic hardening; Sec. 5.2: incremental loading).

    In uniaxial strain the plastic flow keeps the fixed direction diag(1, -1/2, -1/2), so with
    S = 2 mu e - 3 mu alpha the stresses are s11 = kappa e + 2 S / 3, s22 = s33 = kappa e - S / 3.
    While loading, S sits on the yield surface (S = sy + H alpha). On unloading alpha stays at
    its largest value and the response is elastic (|S| < sy + H alpha, checked below). On
    reloading the yield surface is met again exactly at the largest strain reached so far and
    the hardening branch continues. So alpha = max(0, (2 mu e_max - sy) / (3 mu + H)) with
    e_max the largest strain so far. A path solver that did not carry the internal variables
    from one increment to the next would return to the yield surface on unloading instead."""
    lam, mu, sy, H = 40.4, 26.9, 0.25, 1.0
    kappa = lam + 2 * mu / 3
    strains = [0.005, 0.01, 0.015, 0.02, 0.018, 0.016, 0.018, 0.02, 0.022, 0.025]
    path = np.zeros((len(strains), 6))
    path[:, 0] = strains
    pm = np.zeros((4, 6), np.uint8)
    ph = phase_table([(lam, mu, sy, H, 1)])
    sbar, iters, res = O.solve_path(pm, ph, path, np.zeros((1, 3), np.int64), tol=1e-10)
    assert np.all(iters == 1)
    emax = 0.0
    for n, e in enumerate(strains):
        emax = max(emax, e)
        alpha = max(0.0, (2 * mu * emax - sy) / (3 * mu + H))
        S = 2 * mu * e - 3 * mu * alpha
        assert abs(S) <= sy + H * alpha + 1e-12          # on or inside the yield surface
        if e < emax:
            assert abs(S) < sy + H * alpha - 1e-3         # unloading is strictly elastic
        assert np.isclose(sbar[n, 0], kappa * e + 2 * S / 3, rtol=1e-12, atol=1e-15), n
        assert np.isclose(sbar[n, 1], kappa * e - S / 3, rtol=1e-12, atol=1e-15), n
        assert np.isclose(sbar[n, 2], kappa * e - S / 3, rtol=1e-12, atol=1e-15), n
    assert np.allclose(res.alpha, alpha, rtol=1e-12)


def _implicit_j2_point(eps, eps_p, alpha, lam, mu, sy, H):
    """One backward-Euler increment of the J2 model at a material point, solved as a nonlinear
    system instead of the closed-form radial return: unknowns sigma (3x3 symmetric, six
    entries) and the plastic multiplier dg >= 0, equations
        sigma = C : (eps - eps_p - dg * n(sigma)),  n = 3/2 dev(sigma) / sigma_eq(sigma)
        sigma_eq(sigma) = sy + H (alpha + dg)
    (Sec. 2: flow normal to the von Mises surface, consistency on yielding). Elastic when the
    trial stress lies inside the surface."""
    from scipy.optimize import fsolve

    C = O.isotropic_stiffness(lam, mu)
    iu = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]

    def to_t(v):
        t = np.zeros((3, 3))
        for a, (i, j) in enumerate(iu):
            t[i, j] = t[j, i] = v[a]
        return t

    def seq_dev(s):
        d = s - np.trace(s) / 3 * np.eye(3)
        return np.sqrt(1.5 * np.sum(d * d)), d

    trial = np.einsum("ijkl,kl->ij", C, eps - eps_p)
    if seq_dev(trial)[0] <= sy + H * alpha:
        return trial, eps_p, alpha

    # unknowns scaled to order one: sigma / sy and dg * mu / sy
    def F(u):
        s, dg = to_t(u[:6]) * sy, u[6] * sy / mu
        q, d = seq_dev(s)
        n = 1.5 * d / q
        r1 = s - np.einsum("ijkl,kl->ij", C, eps - eps_p - dg * n)
        r2 = q - (sy + H * (alpha + dg))
        return np.concatenate([[r1[i, j] for (i, j) in iu], [r2]]) / sy

    u0 = np.concatenate([[trial[i, j] / sy for (i, j) in iu], [0.0]])
    u, info, ok, msg = fsolve(F, u0, xtol=1e-13, full_output=True)
    assert np.max(np.abs(F(u))) < 1e-12, msg
    s, dg = to_t(u[:6]) * sy, u[6] * sy / mu
    q, d = seq_dev(s)
    return s, eps_p + dg * 1.5 * d / q, alpha + dg


def test_homogeneous_j2_non_proportional_path_matches_implicit_integration():
    """Shear first, then normal strain on top (plane strain, eps_33 = 0): the second increment
    starts from the plastic strain the first one left, in a different direction, so the answer
    depends on the committed internal variables. Checked against a backward-Euler integration
    of the J2 model solved as a nonlinear system."""
    lam, mu, sy, H = 40.4, 26.9, 0.25, 1.0
    path = np.array([[0.0, 0.0, 0, 0, 0, 0.01],
                     [0.01, 0.0, 0, 0, 0, 0.01],
                     [0.01, -0.006, 0, 0, 0, 0.004]])
    pm = np.zeros((3, 5), np.uint8)
    ph = phase_table([(lam, mu, sy, H, 1)])
    sbar, iters, res = O.solve_path(pm, ph, path, np.zeros((1, 3), np.int64), tol=1e-10)
    assert np.all(iters == 1)
    eps_p, alpha = np.zeros((3, 3)), 0.0
    for n in range(len(path)):
        s, eps_p, alpha = _implicit_j2_point(O.vec6_to_tensor(path[n]), eps_p, alpha,
                                             lam, mu, sy, H)
        want = O.tensor_to_vec6(s)
        assert np.allclose(sbar[n], want, rtol=1e-9, atol=1e-12), (n, sbar[n], want)
    assert alpha > 0 and np.allclose(res.alpha, alpha, rtol=1e-9)
    assert np.allclose(res.eps_p[0, 0, 0], eps_p, atol=1e-12)


# ----------------------------------------------------------------------------- brute force
def test_reduced_fixed_point_equals_dense_galerkin_solve():
    pm = np.zeros((8, 8), np.uint8)
    pm[2:6, 1:5] = 1
    pm[6, 6] = 1
    ebar = np.array([0.01, -0.002, 0, 0, 0, 0.003])
    pat = O.pattern_adapted(pm, 1, 21)
    r = O.solve(pm, TWO_PHASE, ebar, pat, tol=1e-14, max_iter=20000)
    # dense system: u = M u + b on the non-zero, non-null frequencies (9 comps each)
    g = _as_grid(pm)
    nz, ny, nx = g.shape
    N = g.size
    lam0, mu0 = O.reference_medium(TWO_PHASE, pm)
    q, null = O.wave_vector(pat, (nx, ny, nz))
    G = O.green_operator(q, lam0, mu0).reshape(-1, 9, 9)
    act = ~null & np.any(pat != 0, axis=1)
    P = pat[act]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = np.array([np.exp(-2j * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz)).ravel()
                   for kx, ky, kz in P])                                  # [K', N]
    F, Finv = ph, ph.conj().T / N
    D = np.stack([(O.isotropic_stiffness(TWO_PHASE["lam"][p], TWO_PHASE["mu"][p])
                   - O.isotropic_stiffness(lam0, mu0)).reshape(9, 9) for p in g.ravel()])
    Ga = G[act]
    Kp = len(P)
    M = -np.einsum("kij,kx,xjl,xm->kiml", Ga, F, D, Finv).reshape(Kp * 9, Kp * 9)
    e9 = O.vec6_to_tensor(ebar).reshape(9)
    b = -np.einsum("kij,kx,xjl,l->ki", Ga, F, D, e9).reshape(Kp * 9)
    u = np.linalg.solve(np.eye(Kp * 9) - M, b).reshape(Kp, 3, 3)
    assert np.allclose(r.eps_hat[act], u, atol=1e-13 * N)


def test_warm_start_from_converged_coefficients_is_a_fixed_point():
    pm = centred_disc(16, 0.3)
    ebar = np.array([0.01, 0, 0, 0, 0, 0])
    pat = O.pattern_adapted(pm, 1, 26)
    r = O.solve(pm, TWO_PHASE, ebar, pat, tol=1e-13, max_iter=5000)
    w = O.solve(pm, TWO_PHASE, ebar, pat, tol=1e-10, warm_hat=r.eps_hat)
    assert w.iters == 1 and np.allclose(w.sigma_bar, r.sigma_bar, rtol=1e-11)


def test_full_set_equals_textbook_full_grid_scheme():
    pm = centred_disc(16, 0.3)
    ebar = np.array([0.01, -0.01, 0, 0, 0, 0])
    r = O.solve(pm, TWO_PHASE, ebar, O.pattern_adapted(pm, 1, pm.size), tol=1e-10, max_iter=2000)
    # independent full-grid basic scheme with the normal-vector form of Gamma applied to tau
    lam, mu = TWO_PHASE["lam"][pm], TWO_PHASE["mu"][pm]
    lam0, mu0 = 0.5 * (lam.min() + lam.max()), 0.5 * (mu.min() + mu.max())
    ny, nx = pm.shape
    ky, kx = np.meshgrid(np.fft.fftfreq(ny) * ny, np.fft.fftfreq(nx) * nx, indexing="ij")
    tx, ty = np.pi * kx / nx, np.pi * ky / ny
    qx, qy = 2 * np.sin(tx) * np.cos(ty), 2 * np.sin(ty) * np.cos(tx)
    qn = np.sqrt(qx ** 2 + qy ** 2)
    qn[0, 0] = 1
    n1, n2 = qx / qn, qy / qn
    c = (lam0 + mu0) / (mu0 * (lam0 + 2 * mu0))
    e11 = np.full(pm.shape, ebar[0])
    e22 = np.full(pm.shape, ebar[1])
    e12 = np.zeros(pm.shape)
    for _ in range(2000):
        tr = e11 + e22
        t11 = (lam - lam0) * tr + 2 * (mu - mu0) * e11
        t22 = (lam - lam0) * tr + 2 * (mu - mu0) * e22
        t12 = 2 * (mu - mu0) * e12
        T11, T22, T12 = (np.fft.fft2(a) for a in (t11, t22, t12))
        v1 = T11 * n1 + T12 * n2
        v2 = T12 * n1 + T22 * n2
        nTn = n1 * v1 + n2 * v2
        E11 = -(n1 * v1 / mu0 - c * n1 * n1 * nTn)
        E22 = -(n2 * v2 / mu0 - c * n2 * n2 * nTn)
        E12 = -((n1 * v2 + n2 * v1) / (2 * mu0) - c * n1 * n2 * nTn)
        E11[0, 0], E22[0, 0], E12[0, 0] = ebar[0] * pm.size, ebar[1] * pm.size, 0
        new = [np.real(np.fft.ifft2(a)) for a in (E11, E22, E12)]
        d = np.sqrt(np.mean((new[0] - e11) ** 2 + (new[1] - e22) ** 2 + 2 * (new[2] - e12) ** 2))
        e11, e22, e12 = new
        if d / np.sqrt(2) / 0.01 < 1e-10:
            break
    assert np.allclose(r.eps[0][..., 0, 0], e11, atol=1e-11)
    assert np.allclose(r.eps[0][..., 0, 1], e12, atol=1e-11)


# ----------------------------------------------------------------------------- patterns
def test_adapted_pattern_laminate_matches_dirichlet_kernel():
    nx, w = 32, 7
    pm = np.zeros((4, nx), np.uint8)
    pm[:, :w] = 1
    kx = np.array([i if i <= nx // 2 else i - nx for i in range(nx)])
    amp = np.where(kx == 0, w, np.abs(np.sin(np.pi * kx * w / nx)
                                      / np.where(kx == 0, 1, np.sin(np.pi * kx / nx))))
    aq = np.rint(amp / w * 2.0 ** 30).astype(np.int64)
    # expected order on the axis (k and -k share their amplitude; ties -> |k|^2 -> index)
    order = sorted(range(nx), key=lambda i: (-aq[i], kx[i] ** 2, kx[i] + (nx - 1) // 2))
    for K in (1, 3, 7, 12):
        got = O.pattern_adapted(pm, 1, K)
        assert np.all(got[:, 1] == 0) and np.all(got[:, 2] == 0)
        taken, n = set(), 0
        for i in order:
            if kx[i] in taken:
                continue
            pair = {int(kx[i]), int(-kx[i]) if abs(kx[i]) != nx // 2 else int(kx[i])}
            taken |= pair
            n = len(taken)
            if n >= K:
                break
        assert set(got[:, 0].tolist()) == taken


@pytest.mark.parametrize("shape,K", [((16, 16), 26), ((12, 20), 50), ((6, 8, 10), 40)])
def test_adapted_pattern_structure_and_topk(shape, K):
    if len(shape) == 2:
        pm = random_discs(shape[0], (2.0, 4.0), 0.3, seed=11) if shape[0] == shape[1] else \
            (np.random.default_rng(3).random(shape) < 0.3).astype(np.uint8)
    else:
        pm = (np.random.default_rng(4).random(shape) < 0.3).astype(np.uint8)
    pat = O.pattern_adapted(pm, 1, K)
    g = _as_grid(pm)
    s = {tuple(p) for p in pat}
    assert (0, 0, 0) in s and K <= len(pat) <= K + 1
    nz, ny, nx = g.shape
    sidx = lambda i, n: i if i <= n // 2 else i - n  # noqa: E731
    for kx, ky, kz in s:
        assert (sidx(-kx % nx, nx), sidx(-ky % ny, ny), sidx(-kz % nz, nz)) in s
    # amplitudes by the DFT definition (brute force); chosen >= not chosen (quantisation slack)
    allk = np.array([(sidx(i, nx), sidx(j, ny), sidx(l, nz)) for l in range(nz)
                     for j in range(ny) for i in range(nx)])
    amp = np.abs(brute_forward((g == 1).astype(float)[..., None], allk))[:, 0]
    chosen = np.array([tuple(k) in s for k in allk])
    tol = g.sum() * 2.0 ** -29
    assert amp[chosen].min() >= amp[~chosen].max() - tol


def test_radial_pattern_structure():
    pat = O.pattern_radial((32, 32), 100)
    s = {tuple(p) for p in pat}
    assert (0, 0, 0) in s and 100 <= len(pat) <= 101
    for kx, ky, _ in s:
        c = ((-kx) % 32, (-ky) % 32)
        c = tuple(v if v <= 16 else v - 32 for v in c)
        assert (c[0], c[1], 0) in s
    assert {(k, 0, 0) for k in range(-3, 4)} <= s and {(0, k, 0) for k in range(-3, 4)} <= s


def test_error_measures():
    rng = np.random.default_rng(9)
    sref = rng.standard_normal((1, 4, 4, 3, 3))
    sref = sref + sref.transpose(0, 1, 2, 4, 3)
    sb = O.tensor_to_vec6(sref.reshape(-1, 3, 3).mean(0))
    Ebar, E = O.errors(2 * sref, sref, 2 * sb, sb)
    assert np.isclose(Ebar, 1.0) and np.isclose(E, 1.0)
    assert O.errors(sref, sref, sb, sb) == (0.0, 0.0)


def test_reference_medium_fixes_the_contraction_ratio():
    """Pure shear of a two-phase laminate: with mu0 = (mu_1 + mu_2)/2 the shear error obeys
    e <- -P[(mu - mu0)/mu0 e], a scalar map whose ratio is rho |1 - 2 f|,
    rho = (mu_2 - mu_1)/(mu_1 + mu_2), f = volume fraction of phase 2."""
    pm = laminate((4, 16), (11, 5))
    f = 5 / 16
    ebar = np.array([0, 0, 0, 0, 0, 0.004])
    r = O.solve(pm, TWO_PHASE, ebar, O.pattern_adapted(pm, 1, pm.size), tol=1e-15,
                max_iter=12, keep_history=True)
    mu = TWO_PHASE["mu"]
    rho = (mu[1] - mu[0]) / (mu[0] + mu[1])
    h = np.array(r.history)
    assert np.allclose(h[2:8] / h[1:7], rho * abs(1 - 2 * f), rtol=1e-9)
    assert O.reference_medium(TWO_PHASE, pm) == (0.5 * sum(TWO_PHASE["lam"]), 0.5 * sum(mu))


# ----------------------------------------------------------------------------- compatibility step
def test_compat_step_leaves_a_full_set_solution_unchanged():
    """The converged solution on the full set of frequencies is a fixed point of the full-set
    update, so the compatibility step (one full-set update, Sec. 5.1) must return it unchanged
    (elastic and J2 with frozen internal variables)."""
    from synth.configs import j2_phases
    pm = random_discs(16, (2.0, 4.0), 0.35, seed=3)
    for ph, ebar in ((TWO_PHASE, np.array([0.01, -0.004, 0, 0, 0, 0.003])),
                     (j2_phases(), np.array([0.02, 0, 0, 0, 0, 0.004]))):
        full = O.full_pattern(_as_grid(pm).shape)
        assert len(full) == pm.size
        r = O.solve(pm, ph, ebar, full, tol=1e-13, max_iter=20000)
        assert r.converged
        eps_c, sig_c, sbar_c = O.compat(pm, ph, r.eps, ebar)
        assert np.allclose(eps_c, r.eps, rtol=0, atol=1e-11 * np.abs(r.eps).max())
        assert np.allclose(sbar_c, r.sigma_bar, rtol=1e-10, atol=1e-14)


def test_compat_step_output_is_compatible_with_the_macro_strain():
    """The step's strain field has mean ebar and, at every nonzero frequency with a nonzero
    wave vector, lies in the range of the compatible projector Gamma0 C0 (closed form above):
    eps^(xi) = sym(q (x) u) for some u."""
    pm = centred_disc(12, 0.3)
    ebar = np.array([0.01, 0.003, 0, 0, 0, -0.002])
    pat = O.pattern_adapted(pm, 1, 19)
    r = O.solve(pm, TWO_PHASE, ebar, pat, tol=1e-10)
    eps_c, _, _ = O.compat(pm, TWO_PHASE, r.eps, ebar)
    assert np.allclose(eps_c.reshape(-1, 3, 3).mean(axis=0), O.vec6_to_tensor(ebar), atol=1e-15)
    g = _as_grid(pm)
    full = O.full_pattern(g.shape)
    q, null = O.wave_vector(full, (g.shape[2], g.shape[1], g.shape[0]))
    lam0, mu0 = O.reference_medium(TWO_PHASE, pm)
    Gcf = gamma_closed_form(q, lam0, mu0)
    eh = O.forward_reduced(eps_c, full)
    C0 = O.isotropic_stiffness(lam0, mu0)
    for m in range(len(full)):
        if null[m] or not np.any(full[m]):
            continue
        proj = np.einsum("ijab,abkl,kl->ij", Gcf[m], C0, eh[m])
        assert np.allclose(proj, eh[m], atol=1e-12 * max(1.0, np.abs(eh).max()))


def test_compat_step_on_a_laminate_gives_the_closed_form():
    """For layers normal to x the reduced solution on the k_y = 0 axis is already exact; the
    compatibility step must reproduce the laminate closed form (uniform sigma_11, sigma_12)."""
    pm = laminate((6, 16), (5, 11))
    ebar = np.array([0.01, -0.004, 0, 0, 0, 0.003])
    pat = O.pattern_adapted(pm, 1, 16)
    r = O.solve(pm, TWO_PHASE, ebar, pat, tol=1e-13, max_iter=5000)
    _, sig_c, _ = O.compat(pm, TWO_PHASE, r.eps, ebar)
    f = np.array([np.mean(pm == 0), np.mean(pm == 1)])
    s11, s12, _, _, _ = laminate_closed_form(TWO_PHASE["lam"], TWO_PHASE["mu"], f, ebar)
    assert np.allclose(sig_c[..., 0, 0], s11, rtol=1e-10)
    assert np.allclose(sig_c[..., 0, 1], s12, rtol=1e-10)


# ----------------------------------------------------------------------------- mixed control
def test_mixed_control_homogeneous_plane_strain_uniaxial_stress():
    """One phase, eps_11 = e prescribed, sigma_22 = sigma_12 = 0 prescribed (plane strain):
    eps_22 = -lam / (lam + 2 mu) e and sigma_11 = 4 mu (lam + mu) / (lam + 2 mu) e."""
    lam, mu, e = 3.0, 1.7, 0.01
    pm = np.zeros((6, 8), np.uint8)
    ph = phase_table([(lam, mu, 0, 0, 0)])
    r = O.solve(pm, ph, np.array([e, 0, 0, 0, 0, 0]), np.zeros((1, 3), np.int64), tol=1e-13,
                control=[0, 1, 0, 0, 0, 1])
    assert np.isclose(r.macro_strain[1], -lam / (lam + 2 * mu) * e, rtol=1e-12)
    assert np.isclose(r.sigma_bar[0], 4 * mu * (lam + mu) / (lam + 2 * mu) * e, rtol=1e-12)
    assert abs(r.sigma_bar[1]) < 1e-14 and abs(r.sigma_bar[5]) < 1e-14


def test_mixed_control_laminate_closed_form():
    """Layers normal to x with sigma_11 = s and sigma_12 = t prescribed, eps_22 = e22 prescribed:
    sigma_11 and sigma_12 are uniform, eps_22 = e22 in every layer, so eps_11 of phase p is
    (s - lam_p e22) / (lam_p + 2 mu_p) and eps_12 is t / (2 mu_p); the macro strain is their
    volume average (the Reuss side of the laminate)."""
    pm = laminate((6, 16), (5, 11))
    s, t, e22 = 0.4, -0.05, -0.002
    pat = O.pattern_adapted(pm, 1, 16)
    r = O.solve(pm, TWO_PHASE, np.array([s, e22, 0, 0, 0, t]), pat, tol=1e-13, max_iter=20000,
                control=[1, 0, 0, 0, 0, 1])
    f = np.array([np.mean(pm == 0), np.mean(pm == 1)])
    lam, mu = TWO_PHASE["lam"], TWO_PHASE["mu"]
    e11 = np.sum(f * (s - lam * e22) / (lam + 2 * mu))
    e12 = np.sum(f * t / (2 * mu))
    assert np.isclose(r.macro_strain[0], e11, rtol=1e-10)
    assert np.isclose(r.macro_strain[5], e12, rtol=1e-10)
    assert np.isclose(r.macro_strain[1], e22, rtol=1e-14)
    assert np.allclose(r.sigma[..., 0, 0], s, rtol=1e-10)
    assert np.allclose(r.sigma[..., 0, 1], t, rtol=1e-10)


@pytest.mark.parametrize("plastic", [False, True])
def test_mixed_control_recovers_the_strain_controlled_solution(plastic):
    """Prescribing the average stresses a strain-controlled solve produced (and its other strain
    components) must return that solve's macro strain and fields: the fixed point is unique."""
    from synth.configs import j2_phases
    pm = random_discs(16, (2.0, 4.0), 0.35, seed=3)
    ph = j2_phases() if plastic else TWO_PHASE
    ebar = np.array([0.02, -0.004, 0, 0, 0, 0.003])
    pat = O.pattern_adapted(pm, 1, 37)
    a = O.solve(pm, ph, ebar, pat, tol=1e-12, max_iter=20000)
    target = np.array([a.sigma_bar[0], ebar[1], 0, 0, 0, a.sigma_bar[5]])
    b = O.solve(pm, ph, target, pat, tol=1e-12, max_iter=20000, control=[1, 0, 0, 0, 0, 1])
    assert np.allclose(b.macro_strain, ebar, rtol=1e-8, atol=1e-13)
    assert np.allclose(b.eps, a.eps, atol=1e-9 * np.abs(a.eps).max())
