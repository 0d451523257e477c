"""Warm-start network kernels against the FP64 oracle (oracle/mlp.py), the batch hooks against
the oracle's slots, descriptors and coefficients, and what the trained network gains over the
plain start.

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
from oracle.rf_oracle import VOIGT, wave_vector
from synth import random_discs, random_macro_strain
from synth.configs import elastic_phases, k_target

pytestmark = pytest.mark.gpu

TF32_FWD, TF32_GRAD, BF16_FWD = 4e-3, 1e-2, 3e-2


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_net(lib, H=80, maxB=300, seed=1):
    net = lib.WarmStartNet(H, maxB)
    rng = np.random.default_rng(seed)
    parts = []
    for sh in net.shapes():
        fan = sh[0] if len(sh) == 2 else 4.0
        parts.append(rng.standard_normal(sh) / np.sqrt(fan))
    flat = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
    net.rf_mlp_set_params(flat)
    return net, [p.astype(np.float32).astype(np.float64) for p in net.split(flat)]


def dev(a, torch, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def slot_array(g, a, b, w, inv_n, rve, kind):
    """Host rf_slot table as a float32 [n, 8] array (int fields written through a view)."""
    n = len(g)
    arr = np.zeros((n, 8), np.float32)
    arr[:, 0], arr[:, 1] = np.real(g), np.imag(g)
    arr[:, 2], arr[:, 3], arr[:, 4], arr[:, 5] = a, b, w, inv_n
    iv = arr.view(np.int32)
    iv[:, 6], iv[:, 7] = rve, kind
    return arr


def test_forward_matches_oracle(lib):
    import torch
    net, params = make_net(lib)
    B = 300                                # three row tiles, the last one ragged
    X = np.random.default_rng(2).standard_normal((B, M.N_DESC)).astype(np.float32)
    want, _ = M.forward(params, X.astype(np.float64))
    with torch.cuda.stream(net.stream):
        dx = dev(X, torch)
        for prec, tol in (("tf32", TF32_FWD), ("bf16", BF16_FWD)):
            got = net.rf_mlp_forward(dx, prec).cpu().numpy()
            assert got.shape == want.shape
            assert rel(got, want) <= tol, (prec, rel(got, want))
    net.close()


def random_slots(rng, B):
    """Per RVE: GPU slot rows (weights 0, 1, 2) and the oracle's pattern entries they stand for
    (a weight-2 slot is k and -k)."""
    rows, tables, targets, offsets = [], [], [], [0]
    T_rows = []
    for r in range(B):
        n = int(rng.integers(0, 40))
        g = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 0.1
        a = rng.uniform(-0.5, 0.5, n)
        b = rng.uniform(0.02, 0.5, n) * rng.choice([-1, 1], n)
        w = rng.choice([0.0, 1.0, 2.0], n, p=[0.1, 0.2, 0.7])
        t = (rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))) * 0.05
        rows.append(slot_array(g, a, b, w, 1.0 / 256, r, np.where(w == 0, 2, 0)))
        T_rows.append(np.stack([t.real, t.imag], axis=2).reshape(n, 6))
        keep1, keep2 = w >= 1, w == 2
        tables.append(dict(g=np.concatenate([g[keep1], np.conj(g[keep2])]),
                           a=np.concatenate([a[keep1], -a[keep2]]),
                           b=np.concatenate([b[keep1], -b[keep2]]),
                           index=np.arange(keep1.sum() + keep2.sum())))
        targets.append(np.concatenate([t[keep1], np.conj(t[keep2])]))
        offsets.append(offsets[-1] + n)
    return (np.concatenate(rows), np.concatenate(T_rows).astype(np.float32),
            np.array(offsets, np.int64), tables, targets)


def test_gradients_match_oracle(lib):
    import torch
    net, params = make_net(lib, H=48, maxB=64, seed=3)
    rng = np.random.default_rng(4)
    B = 40
    X = rng.standard_normal((B, M.N_DESC)).astype(np.float32)
    E = rng.standard_normal((B, 3))
    E = (E / np.linalg.norm(E, axis=1, keepdims=True)).astype(np.float32)
    slots, T, off, tables, targets = random_slots(rng, B)
    loss_o, grads_o = M.loss_and_grads(params, X.astype(np.float64), tables, targets,
                                       E.astype(np.float64))
    with torch.cuda.stream(net.stream):
        loss = net.rf_mlp_loss_grad(dev(X, torch), dev(E, torch), dev(slots, torch),
                                    dev(off, torch), dev(T, torch))
    g = net.split(net.rf_mlp_get_grads())
    assert abs(loss - loss_o) <= TF32_GRAD * loss_o, (loss, loss_o)
    for name, a, b in zip(["W1", "b1", "W2", "b2", "W3", "b3"], g, grads_o):
        assert rel(a, b) <= TF32_GRAD, (name, rel(a, b))
    net.close()


def test_adam_step_matches_oracle(lib):
    import torch
    net, _ = make_net(lib, H=32, maxB=16, seed=5)
    rng = np.random.default_rng(6)
    B = 16
    X = rng.standard_normal((B, M.N_DESC)).astype(np.float32)
    E = np.tile(np.array([[0.6, 0.0, 0.8]], np.float32), (B, 1))
    slots, T, off, _, _ = random_slots(rng, B)
    p0 = net.split(net.rf_mlp_get_params())
    state = ([np.zeros_like(p, dtype=np.float64) for p in p0],
             [np.zeros_like(p, dtype=np.float64) for p in p0], 0)
    p = [q.astype(np.float64) for q in p0]
    with torch.cuda.stream(net.stream):
        d = [dev(X, torch), dev(E, torch), dev(slots, torch), dev(off, torch), dev(T, torch)]
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


def slot_keys(slots, pm):
    ny, nx = pm.shape
    return [(int(round(s[2] * nx)), int(round(s[3] * ny))) for s in slots]


def test_batch_descriptors_slots_and_coefficients_match_oracle(lib):
    import torch
    pms, macros = population(6)
    pms[3] = np.ascontiguousarray(pms[3][:15])           # a rectangular cell with an odd side
    pms[4] = random_discs(32, (2.0, 6.0), 0.35, seed=9)
    # FFT sides on both axes, Ny != Nx (the y transform by FFT with its own twiddles)
    pms[5] = np.ascontiguousarray(random_discs(48, (2.0, 6.0), 0.3, seed=11)[:24])
    pats = [O.pattern_adapted(pm, 1, k_target(0.08, pm.size)) for pm in pms]
    ph = elastic_phases()
    net = lib.WarmStartNet(16, 8)
    with torch.cuda.stream(net.stream):
        b = lib.BatchSolver(pms, ph, pats, stream=net.stream.cuda_stream, tol=0.0, max_iter=6)
        out = b.rf_batch_solve(macros)
        ns, off = b.rf_batch_slots()
        x, slots = b.rf_batch_descriptors(1, rve_base=10)
        c = b.rf_batch_reduced_strain()
        t, e = net.rf_mlp_targets(dev(macros, torch, torch.float64), slots,
                                  dev(off, torch), c)
        x, slots, c = x.cpu().numpy(), slots.cpu().numpy(), c.cpu().numpy()
        t, e = t.cpu().numpy(), e.cpu().numpy()
    b.close()
    net.close()
    assert np.all(out["iters"] == 6) and off[-1] == ns == len(slots)
    for i, (pm, pat) in enumerate(zip(pms, pats)):
        ny, nx = pm.shape
        xo = M.descriptors(pm, 1, pat)
        assert np.abs(x[i] - xo).max() <= 2e-5, (i, np.abs(x[i] - xo).max())
        rows = slots[off[i]:off[i + 1]]
        assert np.all(rows.view(np.int32)[:, 6] == 10 + i)
        keys = slot_keys(rows, pm)
        pat = np.asarray(pat)
        half = [(int(kx), int(ky)) for kx, ky, _ in pat if kx >= 0]
        assert sorted(keys) == sorted(half)
        G = np.fft.fft2((pm == 1).astype(float)) / pm.size
        gam = np.array([G[ky % ny, kx % nx] for kx, ky in keys])
        assert np.abs(rows[:, 0] + 1j * rows[:, 1] - gam).max() <= 2e-6
        _, null = wave_vector(pat, (nx, ny, 1), "rotated")
        nulls = {(int(kx), int(ky)) for (kx, ky, _), z in zip(pat, null) if z}
        for (kx, ky), row in zip(keys, rows):
            self_conj = kx == 0 or 2 * kx == nx
            want_w = 0 if (kx == 0 and ky == 0) or (kx, ky) in nulls else (1 if self_conj else 2)
            assert row[4] == want_w and np.isclose(row[5], 1 / pm.size)
        r = O.solve(pm, ph, macros[i], pat, tol=0.0, max_iter=6)
        pos = {(int(kx), int(ky)): j for j, (kx, ky, _) in enumerate(pat)}
        want = np.array([[r.eps_hat[pos[k], p, q] for (p, q) in ((0, 0), (1, 1), (0, 1))]
                         for k in keys])
        got = c[off[i]:off[i + 1], :, 0] + 1j * c[off[i]:off[i + 1], :, 1]
        assert rel(got, want) <= 1e-5, (i, rel(got, want))
        _, en = M.unit_direction(macros[i])
        tw = (want / (pm.size * en)) * (rows[:, 4] > 0)[:, None]
        tg = t[off[i]:off[i + 1]].reshape(-1, 3, 2)
        assert rel(tg[..., 0] + 1j * tg[..., 1], tw) <= 1e-5
        assert np.allclose(e[i], M.unit_direction(macros[i])[0], rtol=1e-6)


def test_predicted_warm_start_matches_oracle(lib):
    import torch
    pms, macros = population(6, seed0=900)
    pats = [O.pattern_adapted(pm, 1, k_target(0.08, pm.size)) for pm in pms]
    net, params = make_net(lib, H=64, maxB=4, seed=11)   # B > max_batch: chunked inference
    with torch.cuda.stream(net.stream):
        b = lib.BatchSolver(pms, elastic_phases(), pats, stream=net.stream.cuda_stream)
        _, off = b.rf_batch_slots()
        x, slots = b.rf_batch_descriptors(1)
        w = net.rf_mlp_predict_warm(x, dev(macros, torch, torch.float64), slots,
                                    dev(off, torch)).cpu().numpy()
        xh, sh = x.cpu().numpy(), slots.cpu().numpy()
    b.close()
    net.close()
    O_out, _ = M.forward(params, xh.astype(np.float64))
    for i, pm in enumerate(pms):
        rows = sh[off[i]:off[i + 1]]
        reg = rows[:, 4] > 0
        st = dict(g=(rows[reg, 0] + 1j * rows[reg, 1]).astype(complex),
                  a=rows[reg, 2].astype(float), b=rows[reg, 3].astype(float))
        e, en = M.unit_direction(macros[i])
        want = M.head(O_out[i], st, e) * pm.size * en
        got = w[off[i]:off[i + 1]][reg]
        assert rel(got[..., 0] + 1j * got[..., 1], want) <= BF16_FWD
        assert np.all(w[off[i]:off[i + 1]][~reg] == 0)


def test_device_warm_start_equals_host_warm_start(lib):
    import torch
    pms, macros = population(4, seed0=800)
    pats = [O.pattern_adapted(pm, 1, k_target(0.08, pm.size)) for pm in pms]
    ph = elastic_phases()
    host = []
    net = lib.WarmStartNet(16, 4)
    with torch.cuda.stream(net.stream):
        b = lib.BatchSolver(pms, ph, pats, stream=net.stream.cuda_stream, tol=1e-6,
                            max_iter=2000)
        ns, off = b.rf_batch_slots()
        _, slots = b.rf_batch_descriptors(1)
        slots = slots.cpu().numpy()
        dw = np.zeros((ns, 3, 2), np.float32)
        for i, (pm, pat) in enumerate(zip(pms, pats)):
            r = O.solve(pm, ph, macros[i], pat, tol=1e-9, max_iter=3000)
            w = np.zeros((len(pat), 6, 2), np.float32)
            for a_, (p, q) in enumerate(VOIGT):
                w[:, a_, 0] = r.eps_hat[:, p, q].real
                w[:, a_, 1] = r.eps_hat[:, p, q].imag
            host.append(w)
            pos = {(int(kx), int(ky)): j for j, (kx, ky, _) in enumerate(pat)}
            for k, s in zip(slot_keys(slots[off[i]:off[i + 1]], pm), range(off[i], off[i + 1])):
                dw[s] = w[pos[k]][[0, 1, 5]]
        a = b.rf_batch_solve(macros, warm=host)
        d = b.rf_batch_solve_warm(macros, dev(dw, torch))
    b.close()
    net.close()
    assert np.array_equal(a["iters"], d["iters"]) and np.all(d["iters"] <= 2)
    assert np.array_equal(a["sigma_bar"], d["sigma_bar"])


def test_learned_warm_start_cuts_iterations(lib):
    """Train on solver-generated solutions of 32^2 fibre RVEs, then solve held-out RVEs from
    the network's prediction: fewer updates, the same answers (within the tolerance's reach)."""
    from paper_2103_10203_gb300 import warmstart as W
    ph = elastic_phases()
    pms, macros = W.population(range(20000, 24096), side=32, r_range=(2.0, 6.0), workers=8)
    pats = W.patterns(pms, 0.05)
    net = lib.WarmStartNet(256, 256)
    net.rf_mlp_set_params(W.init_params(net, 0))
    ds = W.generate(net, pms, macros, pats, ph, chunk=4096)
    losses = W.train(net, ds, epochs=30, batch=64, lr=1e-3, lr_final=2e-5)
    assert losses[-1] < 0.5 * losses[0], losses
    tp, tm = W.population(range(30000, 30512), side=32, r_range=(2.0, 6.0))
    tpat = W.patterns(tp, 0.05)
    res = W.evaluate(net, tp, tm, tpat, ph)
    net.close()
    print("plain", res["plain"]["iters_mean"], "learned", res["learned"]["iters_mean"])
    assert res["plain"]["converged"] and res["learned"]["converged"]
    assert res["learned"]["iters_mean"] <= res["plain"]["iters_mean"] - 0.4, \
        (res["plain"]["iters_mean"], res["learned"]["iters_mean"])
    # same fixed point: the stress averages agree to within what tol 1e-6 leaves open
    sp, sl = res["plain"]["sigma_bar"], res["learned"]["sigma_bar"]
    assert np.max(np.abs(sp - sl)) <= 1e-4 * np.max(np.abs(sp))
    # descriptors computed once for the RVE set: the same warm start, the same solves
    assert np.array_equal(res["learned_cached"]["iters"], res["learned"]["iters"])
    assert np.array_equal(res["learned_cached"]["sigma_bar"], sl)
