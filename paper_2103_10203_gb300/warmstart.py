"""Learned warm start for batched reduced-frequency solves (include/rf_mlp.h).

Pipeline, all arithmetic in librf.so's kernels (this module only moves arguments):
  1. population: seeded fibre RVEs (synth) and their adapted patterns (rf_pattern_adapted),
  2. training data: the batched solver converges every RVE (rf_batch_solve);
     rf_batch_descriptors and rf_batch_reduced_strain export network inputs, slot tables and
     converged coefficients, and rf_mlp_targets scales them into targets,
  3. training: Adam on minibatches of RVEs (rf_mlp_train_step, TF32 tensor-core GEMMs),
  4. use: rf_batch_descriptors -> rf_mlp_predict_warm (BF16 GEMMs) -> rf_batch_solve_warm.
The convergence measure still decides when a warm-started solve stops, so its answer is the
plain solve's answer to within the tolerance; only the iteration count changes. Batches,
torch tensors and the network share the network's stream, so device buffers pass between them
in stream order.
"""

from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import time

import numpy as np

from . import rf


def _rve(args):
    seed, side, r_range, vf_range = args
    from synth import random_discs, random_macro_strain
    rng = np.random.Generator(np.random.PCG64(seed))
    vf = float(rng.uniform(*vf_range))
    return random_discs(side, r_range, vf, seed), random_macro_strain(seed + 1, 2)


def population(seeds, side=128, r_range=(8.0, 24.0), vf_range=(0.2, 0.5), workers=0):
    """Phase maps and macroscopic strains of fibre RVEs (for side 128 and the default ranges,
    the 128^2 warm-start population: seed i gives the same RVE as synth's make_config('c5',
    index=i)). workers > 1 draws them in a spawn-started process pool."""
    jobs = [(int(s), side, tuple(r_range), tuple(vf_range)) for s in seeds]
    if workers > 1 and len(jobs) > 64:
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            out = list(ex.map(_rve, jobs, chunksize=64))
    else:
        out = [_rve(j) for j in jobs]
    return [o[0] for o in out], np.array([o[1] for o in out])


def patterns(phase_maps, ratio=0.05, inclusion_phase=1):
    """Adapted patterns (Sec. 4) with K = ceil(ratio N) for every RVE (host arrays)."""
    from synth.configs import k_target
    return [rf.rf_pattern_adapted(pm, inclusion_phase, k_target(ratio, pm.size))
            for pm in phase_maps]


class Dataset:
    """Network inputs x [n][48], unit directions e [n][3], slot table slots [slots][8], per-RVE
    slot offsets [n + 1] (int64), targets t [slots][6] (torch CUDA tensors), plus the plain
    solves' iteration counts."""

    def __init__(self, x, e, slots, offsets, t, iters):
        self.x, self.e, self.slots, self.offsets, self.t = x, e, slots, offsets, t
        self.iters = iters

    def __len__(self):
        return self.x.shape[0]


def generate(net, phase_maps, macros, pats, phases, tol=1e-6, max_iter=2000, chunk=4096,
             inclusion_phase=1):
    """Training data from converged batched solves, `chunk` RVEs per batch."""
    import torch
    with torch.cuda.stream(net.stream):
        return _generate(net, phase_maps, macros, pats, phases, tol, max_iter, chunk,
                         inclusion_phase, net.stream.cuda_stream)


def _generate(net, phase_maps, macros, pats, phases, tol, max_iter, chunk, inclusion_phase,
              stream):
    import torch
    xs, es, sls, offs, ts, its = [], [], [], [], [], []
    base = 0
    for c0 in range(0, len(phase_maps), chunk):
        sl = slice(c0, c0 + chunk)
        b = rf.BatchSolver(phase_maps[sl], phases, pats[sl], stream=stream, tol=tol,
                           max_iter=max_iter, transform="fft")
        m = np.asarray(macros[sl])
        out = b.rf_batch_solve(m)
        x, slots = b.rf_batch_descriptors(inclusion_phase, rve_base=c0)
        coeffs = b.rf_batch_reduced_strain()
        _, off = b.rf_batch_slots()
        d_off = torch.as_tensor(off, dtype=torch.int64, device="cuda")
        d_macro = torch.as_tensor(m, dtype=torch.float64, device="cuda")
        t, e = net.rf_mlp_targets(d_macro, slots, d_off, coeffs)
        torch.cuda.synchronize()
        b.close()
        xs.append(x)
        es.append(e)
        sls.append(slots)
        ts.append(t)
        offs.append(off[:-1] + base)
        base += int(off[-1])
        its.append(out["iters"])
    offs.append(np.array([base], np.int64))
    d_offsets = torch.as_tensor(np.concatenate(offs), dtype=torch.int64, device="cuda")
    return Dataset(torch.cat(xs), torch.cat(es), torch.cat(sls), d_offsets, torch.cat(ts),
                   np.concatenate(its))


def init_params(net, seed=0, out_scale=0.1):
    """LeCun-normal weights (variance 1 / fan_in; the output layer scaled by out_scale), zero
    biases, as one flat float32 array."""
    rng = np.random.default_rng(seed)
    parts = []
    shapes = net.shapes()
    for i, sh in enumerate(shapes):
        if len(sh) == 2:
            w = rng.standard_normal(sh) / np.sqrt(sh[0])
            parts.append(w * (out_scale if i == len(shapes) - 2 else 1.0))
        else:
            parts.append(np.zeros(sh))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def train(net, ds, epochs=40, batch=64, lr=1e-3, lr_final=3e-5, seed=0, log=None):
    """Adam over minibatches of consecutive RVEs (the population is already in random order;
    each epoch starts at a different offset), learning rate decayed geometrically to lr_final.
    Returns the per-epoch mean training loss (sampled)."""
    import torch
    n = len(ds)
    batch = min(batch, n, net.dims["max_batch"])
    torch.cuda.current_stream().synchronize()
    steps = max(1, n // batch)
    total = epochs * steps
    losses = []
    rng = np.random.default_rng(seed)
    k = 0
    for ep in range(epochs):
        off = int(rng.integers(0, n - steps * batch + 1)) if n > steps * batch else 0
        acc, cnt = 0.0, 0
        for s in range(steps):
            a = off + s * batch
            rate = lr * (lr_final / lr) ** (k / max(1, total - 1))
            want = s == steps - 1 or s % 32 == 0
            loss = net.rf_mlp_train_step(ds.x[a:a + batch], ds.e[a:a + batch], ds.slots,
                                         ds.offsets[a:a + batch + 1], ds.t, rate, want_loss=want)
            if want:
                acc += loss
                cnt += 1
            k += 1
        losses.append(acc / max(cnt, 1))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4e}")
    torch.cuda.synchronize()
    return losses


def evaluate(net, phase_maps, macros, pats, phases, tol=1e-6, max_iter=2000, inclusion_phase=1,
             repeats=1):
    """Plain vs learned-warm batched solves of the same RVEs; times (CUDA events on the batch
    stream) include the descriptors and the network inference for the learned start."""
    import torch
    with torch.cuda.stream(net.stream):
        return _evaluate(net, phase_maps, macros, pats, phases, tol, max_iter, inclusion_phase,
                         repeats)


def _evaluate(net, phase_maps, macros, pats, phases, tol, max_iter, inclusion_phase, repeats):
    import torch
    stream = net.stream.cuda_stream
    b = rf.BatchSolver(phase_maps, phases, pats, stream=stream, tol=tol, max_iter=max_iter,
                       transform="fft")
    m = np.asarray(macros)
    d_macro = torch.as_tensor(m, dtype=torch.float64, device="cuda")
    _, off = b.rf_batch_slots()
    d_off = torch.as_tensor(off, dtype=torch.int64, device="cuda")
    vox = np.array([pm.size for pm in phase_maps], dtype=np.float64)
    st = net.stream
    res = {}
    # learned_cached: the descriptors depend on the microstructure and pattern only, so an
    # FE-FFT caller that solves the same RVEs again at new macroscopic strains computes them
    # once; that mode times the network, the warm projection and the solve
    for mode in ("plain", "learned", "learned_cached"):
        ms = []
        if mode == "learned_cached":
            x, slots = b.rf_batch_descriptors(inclusion_phase)
        for _ in range(repeats):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(st)
            if mode == "plain":
                out = b.rf_batch_solve(m)
            else:
                if mode == "learned":
                    x, slots = b.rf_batch_descriptors(inclusion_phase)
                w = net.rf_mlp_predict_warm(x, d_macro, slots, d_off)
                out = b.rf_batch_solve_warm(m, w)
            e1.record(st)
            e1.synchronize()
            wall = time.perf_counter() - t0
            ms.append(e0.elapsed_time(e1))
        its = out["iters"].astype(np.int64)
        res[mode] = dict(ms=float(np.median(ms)), wall_s=wall, iters_mean=float(its.mean()),
                         iters_max=int(its.max()), iters=its, sigma_bar=out["sigma_bar"],
                         converged=bool(out["converged"]),
                         voxel_iterations=float(np.sum(its * vox)))
    res["launches"] = b.rf_batch_info()["kernel_launches"]
    b.close()
    return res
