"""Reduced-frequency Moulinec-Suquet solver in float64 (test infrastructure only).

Conventions
-----------
* Grids are arrays of shape (Nz, Ny, Nx), x fastest; 2D problems have Nz = 1 and are plane
  strain (eps_33 = eps_13 = eps_23 = 0; sigma_33 is an output).
* Tensors are full 3x3 arrays on every voxel. Six-vectors use the order (11,22,33,23,13,12)
  with TENSOR (not engineering) shear components.
* A frequency is an integer vector k = (kx, ky, kz) in the signed range (-N_j/2, N_j/2]
  (for even N_j the Nyquist index is +N_j/2). The DFT is
      f^(k) = sum_x f(x) exp(-2 pi i sum_j k_j x_j / N_j),
  the inverse carries 1/N; hence the zero frequency of a field with mean m is N m.
* A sampling pattern (reduced set ^R xi, Sec. 4) is an int array [K, 3] of such vectors,
  containing 0 and closed under k -> -k (mod N).
"""

from __future__ import annotations

import dataclasses

import numpy as np

VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
_EYE = np.eye(3)


# --------------------------------------------------------------------------- helpers
def vec6_to_tensor(v) -> np.ndarray:
    """(11,22,33,23,13,12) tensor components -> symmetric 3x3 (last axis -> last two)."""
    v = np.asarray(v, float)
    t = np.zeros(v.shape[:-1] + (3, 3))
    for a, (i, j) in enumerate(VOIGT):
        t[..., i, j] = v[..., a]
        t[..., j, i] = v[..., a]
    return t


def tensor_to_vec6(t) -> np.ndarray:
    t = np.asarray(t)
    return np.stack([t[..., i, j] for (i, j) in VOIGT], axis=-1)


def _as_grid(phase_map: np.ndarray) -> np.ndarray:
    pm = np.asarray(phase_map)
    if pm.ndim == 2:
        pm = pm[None]
    if pm.ndim != 3:
        raise ValueError("phase map must be 2D (Ny, Nx) or 3D (Nz, Ny, Nx)")
    return pm


def _frob2(t: np.ndarray) -> np.ndarray:
    """Squared Frobenius norm over the last two axes (both shear entries counted)."""
    return np.sum(np.abs(t) ** 2, axis=(-2, -1))


def signed_index(i, n):
    """Array index 0..n-1 -> signed frequency in (-n/2, n/2]."""
    i = np.asarray(i)
    return np.where(i <= n // 2, i, i - n)


def grid_shape_xyz(pm: np.ndarray):
    nz, ny, nx = pm.shape
    return np.array([nx, ny, nz])


def pattern_to_index(pattern: np.ndarray, pm_shape):
    """Pattern [K,3] (kx,ky,kz) -> numpy index tuple into an (Nz, Ny, Nx) FFT array."""
    nz, ny, nx = pm_shape
    p = np.asarray(pattern, np.int64)
    return (p[:, 2] % nz, p[:, 1] % ny, p[:, 0] % nx)


# --------------------------------------------------------------------------- material
def isotropic_stiffness(lam: float, mu: float) -> np.ndarray:
    """C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk) (Sec. 2, linear elastic law)."""
    d = _EYE
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def reference_medium(phases, phase_map, rule: str = "minmax"):
    """Homogeneous reference medium C0 of the basic scheme (Sec. 3).

    The paper asks for the arithmetic average of the spatially varying Lame constants. Reading:
    'minmax' = (min + max) / 2 over the phases present (the choice of the cited basic scheme);
    'volume' = the volume average over voxels. Plastic phases enter with their elastic lam, mu.
    """
    pm = np.asarray(phase_map)
    ids, counts = np.unique(pm, return_counts=True)
    lam = np.asarray(phases["lam"], float)[ids]
    mu = np.asarray(phases["mu"], float)[ids]
    if rule == "minmax":
        return 0.5 * (lam.min() + lam.max()), 0.5 * (mu.min() + mu.max())
    if rule == "volume":
        w = counts / counts.sum()
        return float(np.dot(w, lam)), float(np.dot(w, mu))
    raise ValueError(rule)


def law(eps: np.ndarray, lam, mu, sigma_y0=None, hardening=None, plastic=None,
        eps_p=None, alpha=None):
    """Stress from strain for linear elastic phases and the J2 law with linear isotropic
    hardening (Sec. 2: yield function, associative flow, KKT conditions), as a return map with
    the internal variables (eps_p, alpha = accumulated plastic strain) of the previous
    converged increment held fixed.

    All material arguments are per-voxel arrays broadcastable to eps[..., 0, 0].
    Returns (sigma, eps_p_new, alpha_new, plastic_mask).
    """
    lam = np.asarray(lam, float)[..., None, None]
    mu_ = np.asarray(mu, float)[..., None, None]
    if eps_p is None:
        eps_p = np.zeros_like(eps)
    if alpha is None:
        alpha = np.zeros(eps.shape[:-2])
    eps_e = eps - eps_p
    tr = np.trace(eps_e, axis1=-2, axis2=-1)[..., None, None]
    sig_tr = lam * tr * _EYE + 2.0 * mu_ * eps_e
    if plastic is None or not np.any(plastic):
        return sig_tr, eps_p, alpha, np.zeros(eps.shape[:-2], bool)
    # trial deviatoric stress and von Mises equivalent stress
    p = np.trace(sig_tr, axis1=-2, axis2=-1)[..., None, None] / 3.0
    s = sig_tr - p * _EYE
    seq = np.sqrt(1.5 * _frob2(s))
    sy = np.asarray(sigma_y0, float)
    H = np.asarray(hardening, float)
    phi = seq - (sy + H * alpha)
    yielding = np.asarray(plastic, bool) & (phi > 0.0)
    mu0 = np.asarray(mu, float)
    dgamma = np.where(yielding, phi / np.where(yielding, 3.0 * mu0 + H, 1.0), 0.0)
    safe = np.where(yielding, seq, 1.0)
    flow = 1.5 * s / safe[..., None, None]          # d Phi / d sigma
    sigma = sig_tr - 2.0 * mu_ * dgamma[..., None, None] * flow
    eps_p_new = eps_p + dgamma[..., None, None] * flow
    alpha_new = alpha + dgamma
    # consistency check of the return map (yielded points lie on the updated yield surface)
    if np.any(yielding):
        s_new = sigma - (np.trace(sigma, axis1=-2, axis2=-1)[..., None, None] / 3.0) * _EYE
        seq_new = np.sqrt(1.5 * _frob2(s_new))
        viol = np.abs(seq_new - (sy + H * alpha_new))[yielding]
        scale = np.broadcast_to(sy, yielding.shape)[yielding]
        assert np.all(viol <= 1e-10 * np.maximum(scale, 1e-300) + 1e-14), "return map inconsistent"
    return sigma, eps_p_new, alpha_new, yielding


# --------------------------------------------------------------------------- Green operator
def wave_vector(pattern: np.ndarray, grid_xyz, scheme: str = "rotated"):
    """Wave vector used inside the Green operator, per pattern point (Sec. 3).

    'rotated': first-order finite differences on the rotated stencil (the scheme the paper
    cites against Gibbs oscillations): q_j = 2 sin(t_j) prod_{m != j} cos(t_m), t_j = pi k_j/N_j
    (a common complex phase factor is dropped; it cancels in the operator).
    'continuous': q_j = 2 pi k_j / N_j.
    Returns (q [K,3], null [K]) where null marks xi != 0 whose operator is set to zero
    (q = 0 for rotated; a Nyquist component for continuous).
    """
    k = np.asarray(pattern, float)
    n = np.asarray(grid_xyz, float)
    if scheme == "rotated":
        t = np.pi * k / n
        s, c = np.sin(t), np.cos(t)
        q = np.empty_like(k)
        for j in range(3):
            others = [m for m in range(3) if m != j]
            q[:, j] = 2.0 * s[:, j] * c[:, others[0]] * c[:, others[1]]
        nrm = np.linalg.norm(q, axis=1)
        null = (nrm < 1e-9) & np.any(k != 0, axis=1)
    elif scheme == "continuous":
        q = 2.0 * np.pi * k / n
        ki = np.asarray(pattern, np.int64)
        ni = np.asarray(grid_xyz, np.int64)
        nyq = (ni % 2 == 0) & (ni > 1) & (ki == ni // 2)
        null = np.any(nyq, axis=1)
    else:
        raise ValueError(scheme)
    return q, null


def green_operator(q: np.ndarray, lam0: float, mu0: float) -> np.ndarray:
    """Gamma^0_ijkl(q) of the isotropic reference medium, per row of q [M,3] (Sec. 3, eq. Gamma).

    Built as the paper states it: the acoustic tensor C0_ijkl q_j q_l is inverted to the Green
    function G_ik, and Gamma is the symmetrised product of G with two wave-vector factors,
    Gamma_ijkl = 1/4 (G_jk q_l q_i + G_ik q_l q_j + G_jl q_k q_i + G_il q_k q_j).
    Rows with q = 0 give zeros.
    """
    C0 = isotropic_stiffness(lam0, mu0)
    M = q.shape[0]
    A = np.einsum("ijkl,mj,ml->mik", C0, q, q)
    ok = np.linalg.norm(q, axis=1) > 0
    G = np.zeros((M, 3, 3))
    G[ok] = np.linalg.inv(A[ok])
    Gam = 0.25 * (np.einsum("mjk,ml,mi->mijkl", G, q, q)
                  + np.einsum("mik,ml,mj->mijkl", G, q, q)
                  + np.einsum("mjl,mk,mi->mijkl", G, q, q)
                  + np.einsum("mil,mk,mj->mijkl", G, q, q))
    return Gam


# --------------------------------------------------------------------------- transforms
def forward_reduced(field: np.ndarray, pattern: np.ndarray) -> np.ndarray:
    """Step b): transform of a grid field [Nz,Ny,Nx,...] restricted to the reduced set.

    The full FFT is taken and then restricted, as the paper does (Sec. 4). Returns [K, ...]."""
    idx = pattern_to_index(pattern, field.shape[:3])
    return np.fft.fftn(field, axes=(0, 1, 2))[idx]


def inverse_reduced(coeffs: np.ndarray, pattern: np.ndarray, shape_zyx) -> np.ndarray:
    """Step d): real grid field from coefficients [K, ...] on the reduced set, all other
    frequencies zero. Asserts the imaginary part vanishes (pattern conjugate-closed)."""
    nz, ny, nx = shape_zyx
    coeffs = np.asarray(coeffs)
    full = np.zeros((nz, ny, nx) + coeffs.shape[1:], complex)
    full[pattern_to_index(pattern, shape_zyx)] = coeffs
    f = np.fft.ifftn(full, axes=(0, 1, 2))
    im = np.max(np.abs(f.imag)) if f.size else 0.0
    re = np.max(np.abs(f.real)) if f.size else 0.0
    assert im <= 1e-12 * max(re, 1e-300) + 1e-300, "pattern not conjugate-closed"
    return f.real


# --------------------------------------------------------------------------- mixed control
def stiffness_matrix6(lam, mu) -> np.ndarray:
    """[6, 6] matrix A of the isotropic stiffness on six-vectors (11,22,33,23,13,12) with TENSOR
    shear: sigma_a = sum_b A[a, b] e_b, where a shear entry e_b stands for both eps_kl and eps_lk
    (hence the factor 2 on shear columns)."""
    C = isotropic_stiffness(lam, mu)
    A = np.zeros((6, 6))
    for a, (i, j) in enumerate(VOIGT):
        for b, (k, l) in enumerate(VOIGT):
            A[a, b] = C[i, j, k, l] * (1.0 if k == l else 2.0)
    return A


def mixed_macro_strain(control, target, tau_mean, lam0, mu0, dim) -> np.ndarray:
    """Macroscopic strain E under mixed control (six-vectors, tensor shear). Where control_i = 0
    the strain is prescribed, E_i = target_i; where control_i = 1 the average stress is
    prescribed, and averaging the Lippmann-Schwinger equation (<eps> = E, <sigma> = C0 : E +
    <tau>) gives (C0 : E)_i = target_i - <tau>_i, solved for those E_i with the others held.
    In plane strain (dim 2) E_33 = E_23 = E_13 = 0."""
    control = np.asarray(control, int)
    target = np.asarray(target, float)
    A = stiffness_matrix6(lam0, mu0)
    E = np.where(control == 0, target, 0.0)
    if dim == 2:
        E[2:5] = 0.0
    P = np.flatnonzero(control == 1)
    Q = np.flatnonzero(control == 0)
    if len(P):
        rhs = target[P] - np.real(np.asarray(tau_mean))[P] - A[np.ix_(P, Q)] @ E[Q]
        E[P] = np.linalg.solve(A[np.ix_(P, P)], rhs)
    return E


# --------------------------------------------------------------------------- solver
@dataclasses.dataclass
class SolveResult:
    eps: np.ndarray            # [Nz,Ny,Nx,3,3] converged strain
    sigma: np.ndarray          # [Nz,Ny,Nx,3,3] stress at eps
    sigma_bar: np.ndarray      # (11,22,33,23,13,12) volume average of sigma
    iters: int                 # fixed-point updates performed
    residual: float            # last convergence measure
    converged: bool
    eps_hat: np.ndarray        # [K,3,3] reduced strain coefficients on the pattern
    eps_p: np.ndarray | None   # internal variables after the return map at eps
    alpha: np.ndarray | None
    history: list
    macro_strain: np.ndarray | None = None   # six-vector E = <eps> (mixed control)


def _materials(phases, pm):
    f = lambda name: np.asarray(phases[name], float)[pm]  # noqa: E731
    plastic = np.asarray(phases["plastic"], int)[pm] != 0
    return f("lam"), f("mu"), f("sigma_y0"), f("hardening"), plastic


def _c0_apply(eps, lam0, mu0):
    tr = np.trace(eps, axis1=-2, axis2=-1)[..., None, None]
    return lam0 * tr * _EYE + 2.0 * mu0 * eps


def solve(phase_map, phases, macro_strain, pattern, tol=1e-6, max_iter=1000,
          scheme="rotated", ref="minmax", eps_p=None, alpha=None, eps0=None,
          warm_hat=None, keep_history=False, control=None) -> SolveResult:
    """Reduced fixed-point scheme of Sec. 4 (steps a-d) for one macroscopic strain.

    control   optional six ints: 1 where `macro_strain` holds a prescribed average STRESS
              component instead of a strain component (mixed control for FE-FFT coupling,
              Sec. 1). The zero frequency of every update is then N E with E from
              `mixed_macro_strain` and <tau> = tau^(0) / N; the convergence measure is
              normalised by |E0|, E0 the macro strain of the same rule with <tau> = 0 (also the
              plain start).

    eps0      optional starting strain field (load-path continuation); default eps = ebar.
    warm_hat  optional starting coefficients [K,3,3] on the pattern; they are projected onto
              compatible strains (Gamma0 C0 per frequency) and the zero frequency is set to
              N ebar before the first iteration.
    eps_p, alpha  internal variables of the last converged increment (held fixed).
    The loop runs while the convergence measure (Sec. 3) is >= tol (the printed loop header's
    inequality is read the other way round, since as printed the loop would never start).
    """
    pm = _as_grid(phase_map)
    nz, ny, nx = pm.shape
    N = pm.size
    lam, mu, sy, H, plastic = _materials(phases, pm)
    lam0, mu0 = reference_medium(phases, pm, ref)
    dim = 2 if nz == 1 else 3
    if control is not None:
        target = np.asarray(macro_strain, float)
        E = mixed_macro_strain(control, target, np.zeros(6), lam0, mu0, dim)
    else:
        E = np.asarray(macro_strain, float)
    ebar = vec6_to_tensor(E)
    enorm = np.sqrt(_frob2(ebar))

    pattern = np.asarray(pattern, np.int64)
    is_zero = np.all(pattern == 0, axis=1)
    if is_zero.sum() != 1:
        raise ValueError("pattern must contain the zero frequency exactly once")
    q, null = wave_vector(pattern, (nx, ny, nz), scheme)
    Gam = green_operator(q, lam0, mu0)

    def inverse(coeffs):
        return inverse_reduced(coeffs, pattern, pm.shape)

    if warm_hat is not None:
        w = np.asarray(warm_hat, complex).copy()
        C0 = isotropic_stiffness(lam0, mu0)
        w = np.einsum("kijab,abcd,kcd->kij", Gam, C0, w)
        w[null] = 0.0
        w[is_zero] = N * ebar
        eps = inverse(w)
    elif eps0 is not None:
        eps = np.asarray(eps0, float).reshape(nz, ny, nx, 3, 3).copy()
    else:
        eps = np.broadcast_to(ebar, (nz, ny, nx, 3, 3)).copy()

    history = []
    r = np.inf
    it = 0
    eh = None
    while it < max_iter:
        # a) polarization stress
        sigma, _, _, _ = law(eps, lam, mu, sy, H, plastic, eps_p, alpha)
        tau = sigma - _c0_apply(eps, lam0, mu0)
        # b) transform, restricted to the reduced set
        th = forward_reduced(tau, pattern)
        # c) Lippmann-Schwinger update on the reduced set
        eh = -np.einsum("kijab,kab->kij", Gam, th)
        eh[null] = 0.0
        if control is not None:
            E = mixed_macro_strain(control, target, tensor_to_vec6(th[is_zero][0] / N),
                                   lam0, mu0, dim)
            ebar = vec6_to_tensor(E)
        eh[is_zero] = N * ebar
        # d) back to the grid
        eps_new = inverse(eh)
        # convergence measure: RMS over voxels of the Frobenius norm of the update, / |ebar|
        rms = np.sqrt(np.mean(_frob2(eps_new - eps)))
        r = rms / enorm if enorm > 0 else rms
        eps = eps_new
        it += 1
        if keep_history:
            history.append(r)
        if r < tol:
            break
    sigma, eps_p_new, alpha_new, _ = law(eps, lam, mu, sy, H, plastic, eps_p, alpha)
    sbar = tensor_to_vec6(sigma.reshape(-1, 3, 3).mean(axis=0))
    has_plastic = bool(np.any(plastic))
    return SolveResult(eps=eps, sigma=sigma, sigma_bar=sbar, iters=it, residual=float(r),
                       converged=bool(r < tol), eps_hat=eh,
                       eps_p=eps_p_new if has_plastic else None,
                       alpha=alpha_new if has_plastic else None, history=history,
                       macro_strain=tensor_to_vec6(ebar))


def solve_path(phase_map, phases, path, pattern, tol=1e-6, max_iter=1000, scheme="rotated",
               ref="minmax", fixed_iters=None, control=None):
    """Load path of macroscopic strains path[n] (n = 0..T-1), one increment at a time.

    Internal variables are frozen during the iterations of an increment and committed from the
    return map at its converged strain; increment n starts from eps_{n-1} + (ebar_n - ebar_{n-1}).
    fixed_iters: optional per-increment update counts (tol is then ignored), to replay a path
    iterate by iterate.
    control: optional mixed control (see `solve`); path[n] then holds the targets, and increment
    n starts from eps_{n-1} plus the reference medium's response to the increment of the
    targets: mixed_macro_strain applied (with <tau> = 0) to the strain-target increments and the
    stress-target increments measured from the last homogenised stress (from the zero state
    this is the plain start E0).
    Returns (sigma_bar [T,6], iters [T], last SolveResult); with control, the last result's
    macro_strain holds the macroscopic strain reached at the last increment.
    """
    pm = _as_grid(phase_map)
    path = np.asarray(path, float)
    eps_p = np.zeros(pm.shape + (3, 3))
    alpha = np.zeros(pm.shape)
    prev = np.zeros(6)
    eps = None
    sbar = np.zeros((len(path), 6))
    iters = np.zeros(len(path), int)
    res = None
    prev_s = np.zeros(6)
    if control is not None:
        ctl = np.asarray(control, int)
        lam0, mu0 = reference_medium(phases, pm, ref)
        dim = 2 if pm.shape[0] == 1 else 3
    for n, e in enumerate(path):
        if eps is None:
            eps0 = None
        elif control is None:
            eps0 = eps + vec6_to_tensor(e - prev)
        else:
            incr = np.where(ctl == 1, e - prev_s, e - prev)
            eps0 = eps + vec6_to_tensor(mixed_macro_strain(ctl, incr, np.zeros(6), lam0, mu0,
                                                           dim))
        t_n, m_n = (tol, max_iter) if fixed_iters is None else (0.0, int(fixed_iters[n]))
        res = solve(pm, phases, e, pattern, t_n, m_n, scheme, ref, eps_p=eps_p,
                    alpha=alpha, eps0=eps0, control=control)
        if res.eps_p is not None:
            eps_p, alpha = res.eps_p, res.alpha
        eps = res.eps
        prev = e if control is None else res.macro_strain
        prev_s = res.sigma_bar
        sbar[n] = res.sigma_bar
        iters[n] = res.iters
    return sbar, iters, res


def full_pattern(shape_zyx) -> np.ndarray:
    """Every frequency of the grid (the unreduced set), int [N, 3] as (kx, ky, kz)."""
    kx, ky, kz = _signed_grid(shape_zyx)
    return np.stack([kx.ravel(), ky.ravel(), kz.ravel()], axis=1).astype(np.int64)


def compat(phase_map, phases, eps, macro_strain, scheme="rotated", ref="minmax", eps_p=None,
           alpha=None):
    """Compatibility step (Sec. 5.1): the Lippmann-Schwinger equation solved once on the full set
    of frequencies from the fields of a reduced solve. Reading: one update of the basic scheme
    with every frequency (steps a-d of Sec. 4 with the unreduced set), starting from the reduced
    strain field `eps` [Nz,Ny,Nx,3,3] with the internal variables (eps_p, alpha) held fixed:
        tau = sigma(eps) - C0 : eps,  eps_c^(xi) = -Gamma0(xi) : tau^(xi) (xi != 0),
        eps_c^(0) = N ebar, 0 at null frequencies,
    then sigma_c = sigma(eps_c). Returns (eps_c, sigma_c, sigma_bar_c)."""
    pm = _as_grid(phase_map)
    nz, ny, nx = pm.shape
    N = pm.size
    ebar = vec6_to_tensor(macro_strain)
    lam, mu, sy, H, plastic = _materials(phases, pm)
    lam0, mu0 = reference_medium(phases, pm, ref)
    full = full_pattern(pm.shape)
    q, null = wave_vector(full, (nx, ny, nz), scheme)
    Gam = green_operator(q, lam0, mu0)
    eps = np.asarray(eps, float).reshape(nz, ny, nx, 3, 3)
    sigma, _, _, _ = law(eps, lam, mu, sy, H, plastic, eps_p, alpha)
    tau = sigma - _c0_apply(eps, lam0, mu0)
    th = forward_reduced(tau, full)
    eh = -np.einsum("kijab,kab->kij", Gam, th)
    eh[null] = 0.0
    eh[np.all(full == 0, axis=1)] = N * ebar
    eps_c = inverse_reduced(eh, full, pm.shape)
    sigma_c, _, _, _ = law(eps_c, lam, mu, sy, H, plastic, eps_p, alpha)
    return eps_c, sigma_c, tensor_to_vec6(sigma_c.reshape(-1, 3, 3).mean(axis=0))


# --------------------------------------------------------------------------- patterns
def _signed_grid(shape_zyx):
    nz, ny, nx = shape_zyx
    kz, ky, kx = np.meshgrid(signed_index(np.arange(nz), nz), signed_index(np.arange(ny), ny),
                             signed_index(np.arange(nx), nx), indexing="ij")
    return kx, ky, kz


def _signed_linear(kx, ky, kz, shape_zyx):
    nz, ny, nx = shape_zyx
    hx, hy, hz = (nx - 1) // 2, (ny - 1) // 2, (nz - 1) // 2
    return ((kz + hz) * ny + (ky + hy)) * nx + (kx + hx)


def _conj_signed(k, n):
    return signed_index((-np.asarray(k)) % n, n)


def _select_pairs(order_keys, kx, ky, kz, shape_zyx, k_target):
    """Walk conjugate pairs in the order of `order_keys` (tuple for np.lexsort, last = primary)
    over canonical representatives, adding both members, until >= k_target points."""
    nz, ny, nx = shape_zyx
    lin = _signed_linear(kx, ky, kz, shape_zyx)
    cx, cy, cz = _conj_signed(kx, nx), _conj_signed(ky, ny), _conj_signed(kz, nz)
    clin = _signed_linear(cx, cy, cz, shape_zyx)
    canon = lin <= clin
    size = np.where(lin == clin, 1, 2)
    keys = tuple(np.asarray(k)[canon].ravel() for k in order_keys)
    order = np.lexsort(keys)
    sizes = size[canon].ravel()[order]
    csum = np.cumsum(sizes)
    if k_target > csum[-1]:
        raise ValueError("k_target exceeds the number of frequencies")
    npairs = int(np.searchsorted(csum, k_target) + 1)
    chosen = np.zeros(int(np.prod(shape_zyx)), bool)
    sel_lin = lin[canon].ravel()[order[:npairs]]
    sel_clin = clin[canon].ravel()[order[:npairs]]
    full_lin = lin.ravel()
    pos = np.empty(full_lin.size, np.int64)
    pos[full_lin] = np.arange(full_lin.size)
    chosen[pos[sel_lin]] = True
    chosen[pos[sel_clin]] = True
    flat = np.stack([kx.ravel(), ky.ravel(), kz.ravel()], axis=1)
    pts = flat[chosen]
    return pts[np.argsort(full_lin[chosen])].astype(np.int32)


AMP_BITS = 30


def pattern_adapted(phase_map, inclusion_phase: int, k_target: int) -> np.ndarray:
    """Geometrically adapted sampling pattern (Sec. 4.2; 3D as in Sec. 5.3).

    The geometry becomes the step function g = 1 on the inclusion phase, 0 elsewhere; it is
    transformed, and the frequencies with the largest amplitudes |g^| are kept. Readings where
    the paper is silent: amplitudes are quantised to round(|g^| / |g^(0)| * 2^30) so that
    equal amplitudes tie exactly; ties go to the smaller |k|^2, then the smaller signed linear
    index; k and -k enter together (amplitude taken at the pair's canonical member); pairs are
    added until at least k_target frequencies are held. Output sorted by signed linear index
    (z slowest, x fastest), int32 [K, 3] as (kx, ky, kz).
    """
    pm = _as_grid(phase_map)
    g = (pm == inclusion_phase).astype(float)
    ghat = np.fft.fftn(g)
    amp = np.abs(ghat)
    amax = float(g.sum())
    kx, ky, kz = _signed_grid(pm.shape)
    nz, ny, nx = pm.shape
    # amplitude of each point's canonical pair member, so k and -k carry one value
    lin = _signed_linear(kx, ky, kz, pm.shape)
    cx, cy, cz = _conj_signed(kx, nx), _conj_signed(ky, ny), _conj_signed(kz, nz)
    clin = _signed_linear(cx, cy, cz, pm.shape)
    a_can = np.where(lin <= clin, amp, amp[cz % nz, cy % ny, cx % nx])
    if amax > 0:
        aq = np.rint(a_can / amax * float(1 << AMP_BITS)).astype(np.int64)
    else:
        aq = np.zeros_like(lin)
    k2 = kx.astype(np.int64) ** 2 + ky.astype(np.int64) ** 2 + kz.astype(np.int64) ** 2
    # lexsort: last key is primary -> (-aq, k2, lin)
    return _select_pairs((lin, k2, -aq), kx, ky, kz, pm.shape, k_target)


def _round_half_away(v):
    return np.sign(v) * np.floor(np.abs(v) + 0.5)


def radial_mask(L: int, nx: int, ny: int) -> np.ndarray:
    """Boolean [Ny, Nx] (array index order) of the grid points hit by L equiangular lines
    through the origin at angles pi l / L. Each line is rasterised by stepping one grid unit
    along its dominant axis and rounding (half away from zero) the other coordinate; points
    beyond the signed range are dropped and the index -N/2 is identified with +N/2."""
    mask = np.zeros((ny, nx), bool)
    for l in range(L):
        th = np.pi * l / L
        c, s = np.cos(th), np.sin(th)
        if abs(c) >= abs(s):
            t = np.arange(-(nx // 2), nx // 2 + 1)
            xs, ys = t, _round_half_away(t * (s / c)).astype(np.int64)
        else:
            t = np.arange(-(ny // 2), ny // 2 + 1)
            xs, ys = _round_half_away(t * (c / s)).astype(np.int64), t
        ok = (np.abs(xs) <= nx // 2) & (np.abs(ys) <= ny // 2)
        mask[ys[ok] % ny, xs[ok] % nx] = True
    return mask


def pattern_radial(shape_yx, k_target: int, max_lines: int | None = None) -> np.ndarray:
    """Fixed radial sampling pattern (Sec. 4.1), 2D only. The paper shows it only as a figure:
    reading = the smallest number L of equiangular lines whose rasterised union holds at least
    k_target frequencies, trimmed to k_target (rounded up to whole conjugate pairs) by keeping
    pairs of smaller |k|^2 first, ties by signed linear index. Parity unpinned (no printed
    definition); tests check only its structure."""
    ny, nx = shape_yx
    shape = (1, ny, nx)
    max_lines = max_lines or 4 * max(nx, ny)
    for L in range(1, max_lines + 1):
        mask = radial_mask(L, nx, ny)
        if int(mask.sum()) >= k_target:
            break
    else:
        raise ValueError("k_target not reachable with radial lines")
    kx, ky, kz = _signed_grid(shape)
    on = mask[None]
    k2 = kx.astype(np.int64) ** 2 + ky.astype(np.int64) ** 2
    lin = _signed_linear(kx, ky, kz, shape)
    off = (~on).astype(np.int64)
    return _select_pairs((lin, k2, off), kx, ky, kz, shape, k_target)


# --------------------------------------------------------------------------- errors
def errors(sigma, sigma_ref, sigma_bar, sigma_bar_ref):
    """Macroscopic and microscopic stress errors of Sec. 5 (Frobenius norms).

    Returns (E_bar, E). Voxels with a vanishing reference stress are skipped in E.
    """
    sb = vec6_to_tensor(sigma_bar)
    sr = vec6_to_tensor(sigma_bar_ref)
    Ebar = np.sqrt(_frob2(sb - sr)) / np.sqrt(_frob2(sr))
    num = np.sqrt(_frob2(sigma - sigma_ref)).ravel()
    den = np.sqrt(_frob2(sigma_ref)).ravel()
    ok = den > 1e-300
    E = float(np.sum(num[ok] / den[ok]) / num.size)
    return float(Ebar), E
