#!/usr/bin/env python
"""Throughput of the reduced-frequency solver on the 2D elastoplastic composite workload.

Workload (one step): a 1024 x 1024 periodic composite of random non-overlapping circular
fibres (radius 8-24 voxels, volume fraction 0.4), J2 elastoplastic matrix (E 70 GPa, nu 0.3,
yield 0.25 GPa, H 1 GPa) and elastic fibres (E 400 GPa, nu 0.2), loaded by 20 uniaxial-strain
increments of eps_11 up to 2 %, each solved to a convergence measure below 1e-6 on the
geometrically adapted reduced set with K = 5 % of the frequencies (52429).

Legs:
  value  device-resident: phase map, pattern and state live in HBM; a step is the whole load
         path (rf_reset_path + rf_solve_path). L2 is flushed (256 MB write) before every step,
         outside the timed events. Timed with CUDA events on the solver's stream.
  e2e    the same metric through the C ABI with HOST buffers: pattern generation from the host
         phase map, phase map and pattern upload, load path, homogenised stresses back.
  cpu_baseline  the FP64 oracle on the host cores, a bounded sample of the same workload.
Multi-GPU: independent replicas (one RVE per rank, weak scaling); no data-path collective.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RVE voxel-iterations/s to 1e-6 residual (plain start)"
UNIT = "voxel-iterations/s"
RATIO = 0.05
TOL = 1e-6
MAX_ITER = 20000
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20
TRACE_NOTE = ("mean over the stage's launches of CUDA events recorded around it on the solver's "
              "stream, in a second pass over the same steps (the timed steps run untraced)")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-iters", type=int, default=12, help="oracle updates in the CPU sample")
    p.add_argument("--transform", default="fft", choices=["fft", "dft"])
    p.add_argument("--precision", default="fp32", choices=["fp32", "split_bf16", "split_tf32"])
    p.add_argument("--fft-rows", type=int, default=0,
                   help="c2 FFT mode: rows per row-kernel block (0: autotuned)")
    p.add_argument("--fft-row-blocks", type=int, default=0,
                   help="c2 FFT mode: row-kernel blocks with the rows spread evenly (0: autotuned)")
    p.add_argument("--fft-cols", type=int, default=0,
                   help="c2 FFT mode: columns per column-kernel block (0: autotuned)")
    p.add_argument("--fft-fuse", type=int, default=0, choices=[-1, 0, 1, 2, 3, 4, 5],
                   help="c2 FFT mode column phase: three kernels (-1), one fused kernel (1), "
                        "Green operator inside the inverse y kernel (2), the persistent solve "
                        "(3), the warp-FFT column kernel (4), the persistent solve on the "
                        "warp-FFT passes (5), or timed (0)")
    p.add_argument("--fft-fuse-kx", type=int, default=0,
                   help="c2 FFT mode: kx columns per fused column block (0: autotuned)")
    p.add_argument("--fft-row-warps", type=int, default=0, choices=[-1, 0, 2, 4, 8],
                   help="c2 FFT mode: warps per block of the warp-FFT row kernel (-1: the "
                        "shared-memory row kernel, 0: timed)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "paper", "sweep"],
                   help="c2: 1024^2 J2 load path (the headline line); c3: 128^3 elastic spheres, "
                        "split-BF16 tensor-core transforms; c4: batch of 4096 RVEs of uneven size "
                        "vs per-RVE solves; c5: learned warm start vs plain start; paper: the "
                        "pattern study on the paper-shaped inputs of Sec. 5 (256^2, 256^3); "
                        "sweep: the unfused constitutive sweep alone (4096^2)")
    p.add_argument("--rves", type=int, default=4096, help="c4 / c5: RVEs in the solved batch")
    p.add_argument("--batch-resident", type=int, default=0, choices=[-1, 0, 1],
                   help="c4: RVE-resident solve (1), sweep kernels (-1), or autotuned (0)")
    p.add_argument("--train", type=int, default=50000, help="c5: training RVEs")
    p.add_argument("--epochs", type=int, default=20, help="c5: training epochs")
    p.add_argument("--profile-updates", type=int, default=0,
                   help="run only this many updates of the first increment (for ncu captures)")
    p.add_argument("--no-study", action="store_true",
                   help="c2: skip the pattern study (K = 1/5/10 %%, adapted vs radial vs full set)")
    p.add_argument("--no-sub", action="store_true",
                   help="c2: skip the bounded c4 and c5 summaries folded into the line")
    return p.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def combine_ranks(dist, total_ms, units, device):
    """Whole-job timing of independent replicas: the slowest rank's timed total and the units
    all ranks processed (dist None: one process)."""
    if dist is None:
        return float(total_ms), float(units)
    import torch
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    v = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(v)
    return float(t.item()), float(v.item())


def workload():
    from synth import make_config
    from synth.configs import k_target
    cfg = make_config("c2")
    pm = cfg["phase_map"]
    return cfg, pm, k_target(RATIO, pm.size)


def config_block(pm, K, transform="fft", precision="fp32"):
    return {"workload": "2D 1024x1024 J2 fibre composite (vf 0.4, r 8-24), 20 uniaxial-strain "
                        "increments to 2%, adapted reduced set K=5%",
            "grid": list(pm.shape[::-1]), "K": int(K), "increments": 20, "tol": TOL,
            "transform": transform, "precision": precision,
            "l2": "flushed before every timed step (256 MB write)"}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


# ----------------------------------------------------------------------------- roofline
def stage_work(name, info, shape, transform, nc=3, ns=4):
    """Algorithmic FLOPs and bytes of one launch of a stage (2D workload).

    Bytes are the compulsory device-memory traffic of the launch: phase map and J2 state read
    by the row kernel, line coefficients in and out. FLOPs count the transform arithmetic
    the kernel's algorithm needs (dense DFT: 8 FLOP per complex MAC; FFT: 5 L log2 L per
    complex transform of length L)."""
    import math
    ny, nx = shape
    N = nx * ny
    Kx, Ky = info["Kx"], info["Ky"]
    lines = ny * nc * Kx * 8
    if name == "row":
        byts = N * (1 + 4 * ns) + 2 * lines
        if transform == "fft":
            flops = 2 * (ny * nc / 2) * 5 * nx * math.log2(nx)
        else:
            flops = 8.0 * nc * Kx * N
    elif name in ("inverse_y", "forward_y"):
        byts = (ny + Ky) * nc * Kx * 8
        if transform == "fft":
            flops = nc * Kx * 5 * ny * math.log2(ny)
        else:
            flops = 8.0 * ny * Ky * nc * Kx
    elif name == "column_phase":
        # forward and inverse y transforms of all line columns, Green operator at the pattern
        byts = 2 * ny * nc * Kx * 8 + 2 * info["K_half"] * nc * 8
        flops = 2 * nc * Kx * 5 * ny * math.log2(ny)
    else:
        flops, byts = 0.0, 0.0
    return flops, byts


def sources_sha(files):
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2103_10203_gb300", "csrc")
    for f in files:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, key="dram_bytes_per_launch"):
    """DRAM bytes of `kernel` (per launch, or per `key`) from the committed ncu capture, or None
    when a source file the kernel is built from changed since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as fh:
            k = json.load(fh)["kernels"][kernel]
        if k["sources_sha"] != sources_sha(k["sources"]):
            return None
        return k[key]
    except Exception:
        return None


# ----------------------------------------------------------------------------- CPU oracle
def cpu_sample(pm, phases, pattern, iters):
    """FP64 oracle on the host: `iters` updates of the first solve at eps_11 = 2 % (plastic
    matrix, zero internal variables) on the full 1024^2 grid."""
    import oracle
    macro = np.array([0.02, 0, 0, 0, 0, 0])
    t0c, t0 = time.process_time(), time.perf_counter()
    oracle.solve(pm, phases, macro, pattern, tol=0.0, max_iter=iters)
    wall = time.perf_counter() - t0
    cpu = time.process_time() - t0c
    return {"value": iters * pm.size / wall, "unit": UNIT,
            "cores": max(1, int(round(cpu / wall))), "kind": "oracle",
            "sample": f"{iters} fixed-point updates of the 1024^2 J2 solve at eps_11=2% "
                      f"(oracle, FP64, {wall:.1f} s wall)"}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    cfg, pm, K = workload()
    pat = oracle.pattern_adapted(pm, 1, K)
    its = max(1, args.cpu_iters // 2)
    for _ in range(args.warmup):
        cpu_sample(pm, cfg["phases"], pat, its)
    vals, walls = [], []
    for _ in range(args.steps):
        t = time.perf_counter()
        s = cpu_sample(pm, cfg["phases"], pat, its)
        walls.append(time.perf_counter() - t)
        vals.append(s)
    v = float(np.mean([s["value"] for s in vals]))
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * float(np.mean(walls)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(pm, K), "impl": "reference",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"],
                             "kind": "oracle", "sample": vals[0]["sample"] + " per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- c4 / c5 lines
def _c4_rve(i):
    from synth import make_config
    c = make_config("c4", index=i)
    return c["phase_map"], c["macro"]


def _pool_map(fn, items, workers=16):
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, items, chunksize=32))


def _timed(torch, stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return out, e0.elapsed_time(e1)


def batch_summary(rf, torch, n, steps, warmup, sample_every=8, resident=0):
    """c4: one batched solve of `n` RVEs (sides 64..256, K = 5 %) to 1e-6 vs the same RVEs solved
    one context at a time (every `sample_every`-th RVE, same FP32 FFT transforms)."""
    from synth.configs import elastic_phases, k_target
    rv = _pool_map(_c4_rve, list(range(n)))
    pms = [r[0] for r in rv]
    macros = np.array([r[1] for r in rv])
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    pats = [rf.rf_pattern_adapted(pm, 1, k_target(0.05, pm.size), stream=sh) for pm in pms]
    ph = elastic_phases()
    b = rf.BatchSolver(pms, ph, pats, stream=sh, tol=TOL, max_iter=2000, transform="fft",
                       batch_resident=resident)
    vox = np.array([pm.size for pm in pms], np.float64)
    for _ in range(warmup):
        b.rf_batch_solve(macros)
    l0 = b.rf_batch_info()["kernel_launches"]
    ms, vi = [], 0.0
    with ClockSampler(gpu_id_for(torch, torch.cuda.current_device())) as clk:
        for _ in range(steps):
            out, t = _timed(torch, stream, lambda: b.rf_batch_solve(macros))
            ms.append(t)
            vi += float(np.sum(out["iters"] * vox))
    launches = b.rf_batch_info()["kernel_launches"] - l0
    info = b.rf_batch_info()
    its = out["iters"]
    b.close()
    samp = list(range(0, n, sample_every))
    ctxs = [rf.Solver(pms[i], ph, pattern=pats[i], stream=sh, tol=TOL, max_iter=2000,
                      transform="fft") for i in samp]
    for c, i in zip(ctxs[:8], samp[:8]):
        c.rf_solve(macros[i])

    def solo():
        its_ = 0.0
        for c, i in zip(ctxs, samp):
            its_ += c.rf_solve(macros[i])["iters"] * vox[i]
        return its_
    solo_vi, solo_ms = _timed(torch, stream, solo)
    for c in ctxs:
        c.close()
    total_ms = float(np.sum(ms))
    value = vi / (total_ms / 1e3)
    bytes_per_vox_it = 49.0      # phase 1 B + strain in 12 B + tau out 12 B + line I/O 24 B
    achieved = bytes_per_vox_it * value / 1e9
    hbm = _hbm_peak()
    # DRAM bytes of one solve launch of the resident kernel: the capture's bytes per
    # voxel-iteration (a smaller batch of the same population) times this solve's
    # voxel-iterations
    per_vi = ncu_traffic("kb_resident", "dram_bytes_per_voxel_iteration")
    traffic = (per_vi * vi / steps) if (per_vi is not None and info.get("resident")) else None
    return {"metric": "RVE voxel-iterations/s to 1e-6 residual, batched (plain start)",
            "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": total_ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{n} 2D elastic fibre RVEs, sides U{{64,96,128,192,256}}, "
                                   "vf U[0.2,0.5], r 8-24, K=5% adapted, FP32 (FFT transforms "
                                   "along x and y for sides 2^b and 3*2^b, else pruned DFT)",
                       "voxels": int(vox.sum()), "tol": TOL,
                       "l2": "working set larger than L2"},
            "solves_per_s": n * steps / (total_ms / 1e3),
            "iterations_mean": float(np.mean(its)), "iterations_max": int(np.max(its)),
            "per_rve_launches": {"value": solo_vi / (solo_ms / 1e3), "unit": UNIT,
                                 "sample": f"{len(samp)} of the RVEs (every {sample_every}th), "
                                           "one context each (FFT transforms), solved back to "
                                           "back"},
            "batched_over_per_rve": value / (solo_vi / (solo_ms / 1e3)),
            "gpu_launches": int(launches), "autotuned": info,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "traffic_per_voxel_iteration": (per_vi if traffic is not None
                                                         else None),
                         "kernel": ("kb_resident (a block per RVE runs all its updates)"
                                    if info.get("resident") else
                                    "whole update (the sweep kernels over all RVEs)"),
                         "algorithmic_bytes_per_voxel_iteration": bytes_per_vox_it},
            "clocks": clk.summary()}


def run_batch(args, rf, torch):
    print(json.dumps(batch_summary(rf, torch, args.rves, args.steps, args.warmup,
                                   resident=args.batch_resident)), flush=True)


def _c5_rves(seeds, side=128):
    from paper_2103_10203_gb300 import warmstart as W
    return W.population(seeds, side=side, workers=16)


def learned_summary(rf, torch, n_train, n_test, epochs, steps, single_sample=128):
    """c5: train the warm-start network on `n_train` solver-generated 128^2 solutions, then solve
    `n_test` held-out RVEs from the plain start and from the network's prediction (batched, FP32
    FFT), beside the plain FP32 single-RVE solver and the split-BF16 single-RVE solver on a
    sample of the same RVEs (the forms the batched, warm-started solve is measured against)."""
    from paper_2103_10203_gb300 import warmstart as W
    from synth.configs import elastic_phases
    ph = elastic_phases()
    t0 = time.perf_counter()
    pms, macros = _c5_rves(range(500000, 500000 + n_train))
    pats = W.patterns(pms, 0.05)
    net = rf.WarmStartNet(512, 4096)
    net.rf_mlp_set_params(W.init_params(net, 0))
    ds = W.generate(net, pms, macros, pats, ph, chunk=8192)
    del pms, pats
    t1 = time.perf_counter()
    losses = W.train(net, ds, epochs=epochs, batch=128, lr=1e-3, lr_final=2e-5)
    t2 = time.perf_counter()
    tp, tm = _c5_rves(range(900000, 900000 + n_test))
    tpat = W.patterns(tp, 0.05)
    with ClockSampler(gpu_id_for(torch, torch.cuda.current_device())) as clk:
        res = W.evaluate(net, tp, tm, tpat, ph, repeats=max(1, steps))
    del ds
    launches = net.rf_mlp_launches()
    net.close()
    # single-RVE forms on a sample: plain FP32 FFT and split-BF16 tensor-core transforms
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    samp = list(range(min(single_sample, n_test)))
    single = {}
    for name, kw in (("fp32_fft", dict(transform="fft")),
                     ("split_bf16", dict(transform="dft", precision="split_bf16")),
                     ("split_tf32", dict(transform="dft", precision="split_tf32"))):
        ctxs = [rf.Solver(tp[i], ph, pattern=tpat[i], stream=sh, tol=TOL, max_iter=2000, **kw)
                for i in samp]
        for c, i in zip(ctxs[:4], samp[:4]):
            c.rf_solve(tm[i])
        its = []

        def solo():
            for c, i in zip(ctxs, samp):
                its.append(c.rf_solve(tm[i])["iters"])
        _, t = _timed(torch, stream, solo)
        for c in ctxs:
            c.close()
        single[name] = {"solves_per_s": len(samp) / (t / 1e3), "iterations_mean": float(np.mean(its)),
                        "iterations_max": int(np.max(its)),
                        "sample": f"{len(samp)} held-out RVEs, one context each, back to back"}
    pl, le = res["plain"], res["learned"]
    learned_sps = n_test / (le["ms"] / 1e3)
    return {"metric": "solves/s to 1e-6 residual, learned-warm vs plain start",
            "value": learned_sps, "unit": "solves/s", "n_gpus": 1,
            "steps": steps, "warmup": 0, "ms_per_step": le["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{n_test} held-out 2D 128^2 elastic fibre RVEs (vf "
                                   "U[0.2,0.5], r 8-24), K=5% adapted; network trained on "
                                   f"{n_train} solver-generated solutions",
                       "network": "48 descriptors -> 512 -> 512 -> 243 (27-term transfer "
                                  "expansion per strain/direction pair)",
                       "epochs": epochs, "tol": TOL},
            "plain": {"solves_per_s": n_test / (pl["ms"] / 1e3), "ms": pl["ms"],
                      "iterations_mean": pl["iters_mean"], "iterations_max": pl["iters_max"],
                      "voxel_iterations_per_s": pl["voxel_iterations"] / (pl["ms"] / 1e3)},
            "learned_descriptors_cached": {
                "solves_per_s": n_test / (res["learned_cached"]["ms"] / 1e3),
                "ms": res["learned_cached"]["ms"],
                "speedup": pl["ms"] / res["learned_cached"]["ms"],
                "includes": "BF16 network inference + warm projection; the descriptors (geometry "
                            "and pattern only) computed once for the RVE set, as for RVEs "
                            "solved again at new macroscopic strains"},
            "learned": {"solves_per_s": learned_sps, "ms": le["ms"],
                        "iterations_mean": le["iters_mean"], "iterations_max": le["iters_max"],
                        "voxel_iterations_per_s": le["voxel_iterations"] / (le["ms"] / 1e3),
                        "includes": "features + BF16 network inference + warm projection"},
            "speedup": pl["ms"] / le["ms"],
            "single_rve": single,
            "batched_learned_over_single_fp32": learned_sps / single["fp32_fft"]["solves_per_s"],
            "sigma_bar_max_abs_diff": float(np.max(np.abs(pl["sigma_bar"] - le["sigma_bar"]))),
            "training": {"data_s": t1 - t0, "train_s": t2 - t1, "loss_first": losses[0],
                         "loss_last": losses[-1], "network_launches": int(launches)},
            "clocks": clk.summary()}


def run_learned(args, rf, torch):
    print(json.dumps(learned_summary(rf, torch, args.train, args.rves, args.epochs, args.steps)),
          flush=True)


def _tc_mma_flops(nx, rows, nc, Kx):
    """Tensor-core FLOPs one k_tc_row launch issues (split operands: 3 products per GEMM), from
    the kernel's tiling: 128-wide x slices, R rows per block (tensor-memory limit), Qp = R nc
    padded to 16, the j' = 2 Kx range padded to 128."""
    jt = (2 * Kx + 127) // 128
    R = 16 if nc == 3 else 8
    qp = lambda r: ((r * nc + 15) // 16) * 16
    while R > 1 and qp(R) * (1 + jt) > 512:
        R -= 1
    blocks = ((nx + 127) // 128) * ((rows + R - 1) // R)
    per_block = 3 * 2 * 128 * qp(R) * (jt * 128) * 2      # inverse + forward GEMMs
    return blocks * per_block


def run_3d(args, rf, torch):
    """c3: one elastic 128^3 solve to 1e-6 from the plain start per step, split-BF16 tensor-core
    x transforms (pruned DFT); the FP32 FFT mode timed beside it."""
    from synth import make_config
    cfg = make_config("c3")
    pm, ph, macro = cfg["phase_map"], cfg["phases"], cfg["macro"]
    K = cfg["k_target"]
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    pattern = rf.rf_pattern_adapted(pm, 1, K, stream=sh)
    prec = args.precision if args.precision != "fp32" else "split_bf16"
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(solver, steps, warmup):
        for _ in range(warmup):
            solver.rf_solve(macro)
        ms, its = [], 0
        for s in range(steps):
            flush.fill_(float(s))
            out, t = _timed(torch, stream, lambda: solver.rf_solve(macro))
            ms.append(t)
            its += out["iters"]
        return float(np.sum(ms)), its, out

    if args.profile_updates > 0:
        # a fixed number of traced updates (plain chunk graphs) for profiler captures
        s = rf.Solver(pm, ph, pattern=pattern, stream=sh, tol=0.0, max_iter=args.profile_updates,
                      transform="dft", precision=prec)
        s.rf_set_tracing(True)
        out = s.rf_solve(macro)
        n_launch = s.rf_get_info()["kernel_launches"]
        s.close()
        print(json.dumps({"profile_updates": int(out["iters"]), "kernel_launches": n_launch}))
        return 0
    solver = rf.Solver(pm, ph, pattern=pattern, stream=sh, tol=TOL, max_iter=MAX_ITER,
                       transform="dft", precision=prec)
    info = solver.rf_get_info()
    l0 = info["kernel_launches"]
    with ClockSampler(gpu_id_for(torch, torch.cuda.current_device())) as clk:
        total_ms, its, out = timed(solver, args.steps, args.warmup)
        launches = solver.rf_get_info()["kernel_launches"] - l0
        solver.rf_set_tracing(True)
        solver.rf_reset_stage_times()
        for _ in range(args.steps):
            solver.rf_solve(macro)
        solver.rf_set_tracing(False)
    stage = solver.rf_get_stage_times()
    solver.close()
    fft = rf.Solver(pm, ph, pattern=pattern, stream=sh, tol=TOL, max_iter=MAX_ITER,
                    transform="fft", precision="fp32")
    f_ms, f_its, _ = timed(fft, 1, 1)
    fft.close()
    nz, ny, nx = pm.shape
    N = pm.size
    value = its * N / (total_ms / 1e3)
    row_ms = stage["row"][0] / max(1, stage["row"][1])
    mma = _tc_mma_flops(nx, ny * nz, 6, info["Kx"])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
    peak = peaks["bf16_tflops"] if prec == "split_bf16" else peaks["bf16_tflops"] / 2
    achieved = mma / (row_ms / 1e3) / 1e12
    real = {k: v for k, v in stage.items() if v[1] > 0}
    line = {"metric": "RVE voxel-iterations/s to 1e-6 residual (plain start)", "value": value,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"split_bf16": "bf16x3", "split_tf32": "tf32x3"}[prec],
            "data": "synthetic",
            "config": {"workload": "3D 128^3 elastic spheres (vf 0.25, r 6-12), random symmetric "
                                   "macro strain, adapted reduced set K=2%",
                       "K": int(K), "tol": TOL, "transform": "dft", "precision": prec,
                       "l2": "flushed before every timed step (256 MB write)"},
            "iterations_per_solve": its / args.steps, "gpu_launches": int(launches),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "kernel": "k_tc_row", "launch_ms": row_ms,
                         "mma_flops_per_launch": mma,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS bf16 burst)"
                                        + ("" if prec == "split_bf16" else " / 2 (TF32 nominal ratio)")},
            "stage_share": {k: round(v[0] / sum(x[0] for x in real.values()), 4)
                            for k, v in real.items()},
            "fft_fp32": {"value": f_its * N / (f_ms / 1e3), "unit": UNIT, "iterations": f_its},
            "clocks": clk.summary(),
            "sigma_bar": [float(x) for x in out["sigma_bar"]]}
    print(json.dumps(line), flush=True)


def c2_pattern_study(rf, torch, pm, phases, path, stream, flush, steps=2):
    """Config 2's K in {1, 5, 10} %, adapted vs fixed radial pattern (Sec. 5.2's comparison on
    the 1024^2 J2 composite): time per load path (CUDA events, L2 flushed before each) and the
    Sec. 5 errors of the last increment's stress against the full set of frequencies, before
    and after the compatibility step."""
    from paper_2103_10203_gb300 import sweep
    from synth.configs import k_target
    sh = stream.cuda_stream
    opts = dict(stream=sh, tol=TOL, max_iter=MAX_ITER, transform="fft")
    ref = rf.Solver(pm, phases, pattern=sweep.full_pattern(pm.shape), **opts)
    ref.rf_solve_path(path)
    ref.rf_reset_path()
    flush.fill_(-1.0)
    ref_out, ref_ms = _timed(torch, stream, lambda: ref.rf_solve_path(path))
    rows = []
    try:
        for R in (0.01, 0.05, 0.10):
            K = k_target(R, pm.size)
            for kind in ("adapted", "radial"):
                pat = sweep.pattern(kind, pm, K, stream=sh)
                s = rf.Solver(pm, phases, pattern=pat, **opts)
                s.rf_solve_path(path)               # warm-up: graph built, tiles tuned
                ms, its = [], 0
                for k in range(steps):
                    flush.fill_(float(k))
                    s.rf_reset_path()
                    out, t = _timed(torch, stream, lambda: s.rf_solve_path(path))
                    ms.append(t)
                    its += int(np.sum(out["iters"]))
                eb, e = s.rf_stress_errors(ref)
                s.rf_compat()
                ebc, ec = s.rf_stress_errors(ref)
                s.close()
                rows.append({"ratio": R, "pattern": kind, "K": int(len(pat)),
                             "ms_per_path": float(np.mean(ms)), "updates_per_path": its / steps,
                             "voxel_iterations_per_s": its * pm.size / (float(np.sum(ms)) / 1e3),
                             "Ebar": eb, "E": e, "Ebar_compat": ebc, "E_compat": ec})
    finally:
        ref.close()
    return {"reference": {"K": int(pm.size), "ms_per_path": ref_ms,
                          "updates_per_path": int(np.sum(ref_out["iters"]))},
            "errors": "Sec. 5: Ebar = |sbar - sbar_full| / |sbar_full|, E = mean over voxels of "
                      "|sigma - sigma_full| / |sigma_full|, at the last increment",
            "rows": rows}


def run_paper(args, rf, torch):
    """Pattern study on the paper-shaped inputs (Sec. 5): one inclusion of four shapes (256^2),
    several inclusions elastic and elastoplastic (256^2, 100 increments), one sphere (256^3),
    at the paper's percentages R of frequencies, against the full set of frequencies."""
    from paper_2103_10203_gb300 import sweep
    from synth import make_config
    from synth.configs import PAPER_RATIOS
    sh = torch.cuda.current_stream().cuda_stream
    out = {"metric": "stress errors against the full set of frequencies, adapted vs fixed radial "
                     "pattern (Sec. 5)", "unit": "relative error", "n_gpus": 1,
           "data": "synthetic", "tol": TOL, "studies": {}}
    t0 = time.perf_counter()
    with ClockSampler(gpu_id_for(torch, torch.cuda.current_device())) as clk:
        for shape in ("circle", "annulus", "ellipse", "square"):
            c = make_config("p51", shape=shape)
            rows, ref = sweep.pattern_study(c["phase_map"], c["phases"], PAPER_RATIOS,
                                            macro=c["macro"], stream=sh)
            out["studies"][f"p51_{shape}"] = {"reference": ref, "rows": rows}
        c = make_config("p52")
        rows, ref = sweep.pattern_study(c["phase_map"], c["phases"], PAPER_RATIOS,
                                        macro=c["macro"], stream=sh)
        out["studies"]["p52_elastic"] = {"reference": ref, "rows": rows}
        c = make_config("p52", plastic=True)
        rows, ref = sweep.pattern_study(c["phase_map"], c["phases"], PAPER_RATIOS,
                                        path=c["path"], max_iter=200000, stream=sh)
        out["studies"]["p52_j2_100_increments"] = {"reference": ref, "rows": rows}
        c = make_config("p53")
        rows, ref = sweep.pattern_study(c["phase_map"], c["phases"],
                                        (0.0039, 0.0078, 0.0154, 0.0306, 0.0602),
                                        macro=c["macro"], kinds=("adapted",), stream=sh)
        for r in rows:
            r["ms_per_update"] = 1e3 * r["solve_s"] / max(1, r["iters"])
        ref["ms_per_update"] = 1e3 * ref["solve_s"] / max(1, ref["iters"])
        out["studies"]["p53_sphere_256cube"] = {"reference": ref, "rows": rows}
    j2 = {r["pattern"]: r for r in out["studies"]["p52_j2_100_increments"]["rows"]
          if r["ratio"] == 0.0154}
    out["value"] = j2["adapted"]["E"]
    out["value_is"] = "E of the adapted pattern at R = 1.54 % (several inclusions, J2 matrix)"
    out["radial_E_same_R"] = j2["radial"]["E"]
    out["wall_s"] = time.perf_counter() - t0
    out["clocks"] = clk.summary()
    print(json.dumps(out), flush=True)


def voxel_sweep(rf, torch, reps=20):
    """The unfused constitutive sweep (step a on its own) over the 1024^2 J2 composite tiled 4 x 4
    to 4096^2 (16.8 M voxels, fields far larger than L2): strain planes in, polarization planes
    out, phase map and J2 state read; 41 bytes per voxel. Achieved bandwidth from CUDA events
    over `reps` launches against the measured HBM copy bandwidth."""
    from synth import make_config
    cfg = make_config("c2")
    pm = np.ascontiguousarray(np.tile(cfg["phase_map"], (4, 4)))
    N = pm.size
    # an explicit stream for the solver and the events: the sweep is asynchronous, and a
    # context given the legacy stream makes a stream of its own
    stream = torch.cuda.Stream()
    s = rf.Solver(pm, cfg["phases"], stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        g = torch.Generator(device="cuda").manual_seed(7)
        eps = (torch.rand((3, N), device="cuda", generator=g) - 0.5) * 0.04
        tau = torch.empty_like(eps)
    for _ in range(3):
        s.rf_law_sweep(eps, tau)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        s.rf_law_sweep(eps, tau)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    s.close()
    bpv = 3 * 4 + 1 + 4 * 4 + 3 * 4
    hbm = _hbm_peak()
    achieved = bpv * N / (ms / 1e3) / 1e9
    return {"kernel": "k_law_sweep<3, J2>", "voxels": int(N), "bytes_per_voxel": bpv,
            "launch_ms": ms, "achieved_GBs": achieved, "peak_GBs": hbm, "frac": achieved / hbm,
            "what": "strain 12 B + phase 1 B + J2 state 16 B in, polarization 12 B out per voxel; "
                    "4096^2 tiling of the 1024^2 J2 composite, fields larger than L2"}


def _hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(p))["hbm_gbs"] if os.path.exists(p) else 6800.0


# ----------------------------------------------------------------------------- GPU arm
def main():
    args = parse()
    ws, rank, local = dist_info()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2103_10203_gb300 import rf
    if args.workload == "c3":
        return run_3d(args, rf, torch)
    if args.workload == "c4":
        return run_batch(args, rf, torch)
    if args.workload == "c5":
        return run_learned(args, rf, torch)
    if args.workload == "paper":
        return run_paper(args, rf, torch)
    if args.workload == "sweep":
        print(json.dumps(voxel_sweep(rf, torch)), flush=True)
        return 0

    cfg, pm, K = workload()
    phases, path = cfg["phases"], cfg["path"]
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    pattern = rf.rf_pattern_adapted(pm, 1, K, stream=sh)
    tiles = {}
    if args.transform == "fft":
        tiles = dict(fft_rows=args.fft_rows, fft_cols=args.fft_cols, fft_fuse=args.fft_fuse,
                     fft_row_blocks=args.fft_row_blocks, fft_row_warps=args.fft_row_warps,
                     fft_fuse_kx=args.fft_fuse_kx)
    if args.profile_updates > 0:
        s = rf.Solver(pm, phases, pattern=pattern, stream=sh, tol=0.0,
                      max_iter=args.profile_updates, transform=args.transform,
                      precision=args.precision, **tiles)
        # traced mode replays plain chunk graphs (the same kernels) instead of the graph with
        # a conditional while node, whose kernel nodes a profiler cannot capture one by one
        s.rf_set_tracing(True)
        out = s.rf_solve(path[0])
        n_launch = s.rf_get_info()["kernel_launches"]
        s.close()
        print(json.dumps({"profile_updates": int(out["iters"]), "kernel_launches": n_launch}))
        return 0
    solver = rf.Solver(pm, phases, pattern=pattern, stream=sh, tol=TOL, max_iter=MAX_ITER,
                       transform=args.transform, precision=args.precision, **tiles)
    info = solver.rf_get_info()
    tile_info = {k: info[k] for k in ("fft_rows", "fft_row_threads", "fft_cols",
                                      "fft_col_threads", "fft_fused", "fft_fuse_kx",
                                      "fft_fuse_threads", "fft_row_blocks", "fft_row_warps")} \
        if args.transform == "fft" else None
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        solver.rf_reset_path()
        out = solver.rf_solve_path(path)
        return int(np.sum(out["iters"])), out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = solver.rf_get_info()["kernel_launches"]
    iters, ms_steps, outs = 0, [], []
    with ClockSampler(gpu_id_for(torch, local)) as clk:
        torch.cuda.synchronize()
        for s in range(args.steps):
            flush.fill_(float(s))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            n, out = step()
            e1.record(stream)
            e1.synchronize()
            ms_steps.append(e0.elapsed_time(e1))
            iters += n
            outs.append(out)
        torch.cuda.synchronize()
        launches = solver.rf_get_info()["kernel_launches"] - launches0
        # the same steps again with per-stage CUDA events recorded on the solver's stream
        # (captured into the update graphs); kept out of the timed steps above
        solver.rf_set_tracing(True)
        solver.rf_reset_stage_times()
        for s in range(args.steps):
            flush.fill_(float(s))
            step()
        torch.cuda.synchronize()
        solver.rf_set_tracing(False)
    stage = solver.rf_get_stage_times()
    total_ms, all_iters = combine_ranks(dist, float(np.sum(ms_steps)), iters, "cuda")
    value = all_iters * pm.size / (total_ms / 1000.0)
    solves = ws * args.steps / (total_ms / 1000.0)

    # dominant stage and its roofline
    real = {k: v for k, v in stage.items() if v[1] > 0}
    dom = max(real, key=lambda k: real[k][0])
    dom_ms = real[dom][0] / real[dom][1]
    flops, byts = stage_work(dom, info, pm.shape, args.transform)
    clocks = clk.summary()
    sm_max = clocks["sm_max_mhz"] or 2070.0
    props = torch.cuda.get_device_properties(local)
    kernel_names = {("fft", "row"): "k_fft_row", ("fft", "column_phase"): "k_fft_colphase",
                    ("fft", "inverse_y"): "k_fft_cols",
                    ("fft", "forward_y"): "k_fft_cols", ("dft", "row"): "k_row",
                    ("dft", "inverse_y"): "k_dft_axis", ("dft", "forward_y"): "k_dft_axis"}
    if args.precision != "fp32" and dom == "row":
        kernel_names[("dft", "row")] = "k_tc_row"
    if tile_info and tile_info.get("fft_row_warps"):
        kernel_names[("fft", "row")] = "k_fft_row_w"
    if tile_info and tile_info.get("fft_fused") == 4:
        kernel_names[("fft", "column_phase")] = "k_fft_colphase_w"
    if tile_info and tile_info.get("fft_fused") == 5:
        # the persistent solve on the warp-FFT passes: its row and column phases, each timed up
        # to its grid barrier by global-timer stamps of block 0
        kernel_names[("fft", "row")] = "k_persist_w (row phase)"
        kernel_names[("fft", "column_phase")] = "k_persist_w (column phase)"
    if tile_info and tile_info.get("fft_fused") == 3:
        # the persistent solve: one kernel; its stages are the row and the column phase, each
        # timed up to its grid barrier by global-timer stamps of block 0
        kernel_names[("fft", "row")] = "k_persist2d (row phase)"
        kernel_names[("fft", "column_phase")] = "k_persist2d (column phase)"
    if args.transform == "fft" and dom in ("row", "inverse_y", "forward_y", "column_phase"):
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
        kname = kernel_names[("fft", dom)]
        achieved = byts / (dom_ms / 1e3) / 1e9
        tr = ncu_traffic(kname)
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": tr, "kernel": kname, "stage": dom,
                "launch_ms": dom_ms, "algorithmic_bytes_per_launch": byts,
                "algorithmic_flops_per_launch": flops, "launch_ms_source": TRACE_NOTE,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"}
    elif dom == "row" or dom.endswith("_y"):
        peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        achieved = flops / (dom_ms / 1e3) / 1e12
        kname = kernel_names[("dft", dom)]
        tr = ncu_traffic(kname)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": tr, "kernel": kname, "stage": dom,
                "launch_ms": dom_ms, "algorithmic_flops_per_launch": flops,
                "algorithmic_bytes_per_launch": byts, "launch_ms_source": TRACE_NOTE,
                "peak_source": "FP32 FMA: SMs x 128 lanes x 2 FLOP x max SM clock"}
    else:
        roof = {"bound": "hbm", "achieved": None, "peak": None, "unit": "GB/s", "frac": None,
                "traffic": None, "stage": dom}
    stage_share = {k: round(v[0] / max(1e-9, sum(x[0] for x in real.values())), 4)
                   for k, v in real.items()}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        h2d = pm.nbytes * 2 + len(pattern) * 12 + path.nbytes
        d2h = len(pattern) * 12 + path.shape[0] * (48 + 4 + 8)
        e_iters, e_t = 0, 0.0
        for s in range(args.steps):
            flush.fill_(float(s))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pat = rf.rf_pattern_adapted(pm, 1, K, stream=sh)
            solver.rf_set_phase_map(pm)
            solver.rf_set_pattern(pat)
            out = solver.rf_solve_path(path)
            _ = out["sigma_bar"].sum()
            e_t += time.perf_counter() - t0
            e_iters += int(np.sum(out["iters"]))
        e2e = {"value": e_iters * pm.size / e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # compatibility step on the last solved path (the first call builds the full-set context)
    solver.rf_compat()
    compat_ms = []
    for k in range(3):
        _, t = _timed(torch, stream, solver.rf_compat)
        compat_ms.append(t)
    compat = {"ms": float(np.mean(compat_ms)),
              "what": "one full-set Lippmann-Schwinger update from the reduced solution "
                      "(Sec. 5.1), fields and homogenised stress",
              "per_reduced_update_ms": float(np.sum(ms_steps)) / max(1, iters)}

    sweep_line = None
    try:
        sweep_line = voxel_sweep(rf, torch)
    except Exception as ex:
        sweep_line = {"error": repr(ex)}

    study = None
    if rank == 0 and not args.no_study:
        try:
            study = c2_pattern_study(rf, torch, pm, phases, path, stream, flush)
        except Exception as ex:   # reported, never fatal for the headline line
            study = {"error": repr(ex)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_sample(pm, phases, pattern, args.cpu_iters)

    subs = {}
    if rank == 0 and ws == 1 and not args.no_sub:
        for key, fn in (("c4", lambda: batch_summary(rf, torch, 2048, 2, 3, sample_every=16)),
                        ("c5", lambda: learned_summary(rf, torch, 8192, 1024, 8, 2,
                                                       single_sample=64))):
            try:
                subs[key] = fn()
            except Exception as ex:
                subs[key] = {"error": repr(ex)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "split_bf16": "bf16x3", "split_tf32": "tf32x3"}[args.precision],
                "data": "synthetic",
                "config": config_block(pm, K, args.transform, args.precision),
                "solves_per_s": solves,
                "iterations_per_step": iters / args.steps, "e2e": e2e,
                "gpu_launches": int(launches), "roofline": roof, "stage_share": stage_share,
                "tiles": tile_info,
                "cpu_baseline": cpu, "clocks": clocks, "compat": compat,
                "unfused_voxel_sweep": sweep_line,
                "pattern_study": study,
                "c4_bounded": subs.get("c4"), "c5_bounded": subs.get("c5"),
                "precision": {"fp32": "FP32 transforms and law",
                              "split_bf16": "BF16 hi+lo tensor-core x transforms, FP32 law",
                              "split_tf32": "TF32 hi+lo tensor-core x transforms, FP32 law"}
                [args.precision] + "; FP64 residual and homogenised stress",
                "sigma_bar_final": [float(x) for x in outs[-1]["sigma_bar"][-1]]}
        print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
