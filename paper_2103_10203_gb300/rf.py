"""Python binding of the C ABI in include/rf.h (argument marshalling only).

Every computation happens in librf.so's CUDA kernels. Importing this module loads the
library and raises if it is missing: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librf.so")

RF_OK, RF_NOT_CONVERGED = 0, 1
ERRORS = {-1: "invalid argument", -2: "CUDA error", -3: "non-finite", -4: "diverged",
          -5: "out of memory", -6: "device timeout", -7: "state"}
GREEN = {"rotated": 0, "continuous": 1}
REF = {"minmax": 0, "volume": 1}
PRECISION = {"fp32": 0, "split_bf16": 1, "split_tf32": 2}
TRANSFORM = {"dft": 0, "fft": 1}


class rf_grid(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int32 * 3)]


class rf_phase(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("mu", C.c_double), ("sigma_y0", C.c_double),
                ("hardening", C.c_double), ("plastic", C.c_int32), ("reserved", C.c_int32)]


class rf_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("green", C.c_int32),
                ("ref_medium", C.c_int32), ("precision", C.c_int32), ("check_every", C.c_int32),
                ("transform", C.c_int32), ("fft_rows", C.c_int32), ("fft_cols", C.c_int32),
                ("fft_fuse", C.c_int32), ("fft_fuse_kx", C.c_int32),
                ("fft_row_blocks", C.c_int32), ("wait_limit", C.c_int64),
                ("stall_test", C.c_int32), ("fft_row_warps", C.c_int32),
                ("batch_resident", C.c_int32)]


class rf_info(C.Structure):
    _fields_ = [("K", C.c_int64), ("K_half", C.c_int64), ("Kx", C.c_int32), ("Ky", C.c_int32),
                ("Kz", C.c_int32), ("last_iters", C.c_int32), ("last_residual", C.c_double),
                ("kernel_launches", C.c_int64), ("j2_max_violation", C.c_double),
                ("lambda0", C.c_double), ("mu0", C.c_double), ("fft_rows", C.c_int32),
                ("fft_row_threads", C.c_int32), ("fft_cols", C.c_int32),
                ("fft_col_threads", C.c_int32), ("fft_fused", C.c_int32),
                ("fft_fuse_kx", C.c_int32), ("fft_fuse_threads", C.c_int32),
                ("fft_row_blocks", C.c_int32), ("fft_row_warps", C.c_int32),
                ("reserved", C.c_int32)]


class rf_mlp_dims(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_hidden", C.c_int32), ("n_out", C.c_int32),
                ("max_batch", C.c_int32), ("n_params", C.c_int64), ("adam_steps", C.c_int64)]


class rf_slot(C.Structure):
    _fields_ = [("g_re", C.c_float), ("g_im", C.c_float), ("a", C.c_float), ("b", C.c_float),
                ("weight", C.c_float), ("inv_n", C.c_float), ("rve", C.c_int32),
                ("kind", C.c_int32)]


SLOT_FLOATS = 8   # an rf_slot is 32 bytes: device slot tables are float32 tensors [n][8]


class RFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rf error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    i32, i64, dbl = C.c_int32, C.c_int64, C.c_double
    sig = {
        "rf_create": [C.POINTER(P), C.POINTER(rf_grid), i32, C.POINTER(rf_phase), P,
                      C.POINTER(rf_options), P],
        "rf_set_phase_map": [P, P],
        "rf_set_phase_map_device": [P, P],
        "rf_set_pattern": [P, P, i64],
        "rf_solve": [P, P, P, P, P, P],
        "rf_solve_path": [P, i32, P, P, P, P],
        "rf_reset_path": [P],
        "rf_get_fields": [P, P, P, P],
        "rf_get_reduced_strain": [P, P],
        "rf_get_state": [P, P, C.POINTER(C.c_size_t)],
        "rf_set_state": [P, P, C.c_size_t],
        "rf_get_info": [P, C.POINTER(rf_info)],
        "rf_destroy": [P],
        "rf_compat": [P, P],
        "rf_solve_mixed": [P, P, P, P, P, P, P, P],
        "rf_solve_path_mixed": [P, P, i32, P, P, P, P, P],
        "rf_stress_errors": [P, P, P, P],
        "rf_law_sweep": [P, P, P, P],
        "rf_pattern_adapted": [C.POINTER(rf_grid), P, i32, i64, P, i64, C.POINTER(i64), P],
        "rf_pattern_radial": [C.POINTER(rf_grid), i64, P, i64, C.POINTER(i64), P],
        "rf_pattern_adapted_noalloc": [C.POINTER(rf_grid), P, i32, i64, P, i64, C.POINTER(i64),
                                       P],
        "rf_batch_create": [C.POINTER(P), i32, C.POINTER(rf_grid), P, i32, C.POINTER(rf_phase),
                            P, P, C.POINTER(rf_options), P],
        "rf_batch_solve": [P, P, P, P, P, P, P],
        "rf_batch_info": [P, P, P, P],
        "rf_batch_destroy": [P],
        "rf_batch_mode": [P, P],
        "rf_set_tracing": [P, i32],
        "rf_get_stage_times": [P, P, P],
        "rf_reset_stage_times": [P],
        "rf_mlp_create": [C.POINTER(P), i32, i32, P],
        "rf_mlp_get_dims": [P, C.POINTER(rf_mlp_dims)],
        "rf_mlp_set_params": [P, P],
        "rf_mlp_get_params": [P, P],
        "rf_mlp_get_grads": [P, P],
        "rf_mlp_forward": [P, i32, P, P, i32],
        "rf_mlp_targets": [P, i32, P, P, P, P, P, P],
        "rf_mlp_loss_grad": [P, i32, P, P, P, P, P, C.POINTER(dbl)],
        "rf_mlp_adam": [P, C.c_float],
        "rf_mlp_train_step": [P, i32, P, P, P, P, P, C.c_float, C.POINTER(dbl)],
        "rf_mlp_predict_warm": [P, i32, P, P, P, P, P],
        "rf_mlp_launches": [P, C.POINTER(i64)],
        "rf_mlp_destroy": [P],
        "rf_batch_slots": [P, C.POINTER(i64), P],
        "rf_batch_descriptors": [P, i32, i32, P, P],
        "rf_batch_reduced_strain": [P, P],
        "rf_batch_solve_warm": [P, P, P, P, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.rf_last_error.argtypes = []
    lib.rf_last_error.restype = C.c_char_p
    _ = (dbl,)
    return lib


lib = _load()

# names declared in include/rf.h, for the export check
EXPORTED = ["rf_create", "rf_set_phase_map", "rf_set_phase_map_device", "rf_set_pattern",
            "rf_solve", "rf_solve_path", "rf_reset_path", "rf_get_fields",
            "rf_get_reduced_strain", "rf_get_state", "rf_set_state", "rf_get_info", "rf_destroy",
            "rf_pattern_adapted", "rf_pattern_radial", "rf_last_error", "rf_set_tracing",
            "rf_get_stage_times", "rf_reset_stage_times", "rf_pattern_adapted_noalloc",
            "rf_batch_create", "rf_batch_solve", "rf_batch_info", "rf_batch_destroy",
            "rf_batch_mode", "rf_batch_slots", "rf_batch_descriptors", "rf_batch_reduced_strain",
            "rf_batch_solve_warm", "rf_compat", "rf_stress_errors", "rf_solve_mixed",
            "rf_law_sweep",
            "rf_solve_path_mixed",
            "rf_mlp_create", "rf_mlp_get_dims", "rf_mlp_set_params", "rf_mlp_get_params",
            "rf_mlp_get_grads", "rf_mlp_forward", "rf_mlp_targets", "rf_mlp_loss_grad",
            "rf_mlp_adam", "rf_mlp_train_step", "rf_mlp_predict_warm", "rf_mlp_launches",
            "rf_mlp_destroy"]

STAGES = ["inverse_z", "inverse_y", "row", "forward_y", "forward_z", "green", "column_phase",
          "final"]


def _check(code, allow_nc=True):
    if code == RF_OK or (allow_nc and code == RF_NOT_CONVERGED):
        return code
    raise RFError(code, lib.rf_last_error().decode())


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _dptr(t):
    """Device pointer of a CUDA tensor (or None)."""
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle(stream):
    if stream is None:
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


def make_grid(shape) -> rf_grid:
    """shape (Ny, Nx) or (Nz, Ny, Nx) -> rf_grid."""
    g = rf_grid()
    if len(shape) == 2:
        g.dim, g.n[0], g.n[1], g.n[2] = 2, shape[1], shape[0], 1
    else:
        g.dim, g.n[0], g.n[1], g.n[2] = 3, shape[2], shape[1], shape[0]
    return g


def make_phases(table) -> C.Array:
    arr = (rf_phase * len(table))()
    for i, r in enumerate(table):
        arr[i].lambda_ = float(r["lam"])
        arr[i].mu = float(r["mu"])
        arr[i].sigma_y0 = float(r["sigma_y0"])
        arr[i].hardening = float(r["hardening"])
        arr[i].plastic = int(r["plastic"])
    return arr


def make_options(tol=1e-6, max_iter=1000, green="rotated", ref="minmax", precision="fp32",
                 check_every=0, transform="dft", fft_rows=0, fft_cols=0, fft_fuse=0,
                 fft_fuse_kx=0, fft_row_blocks=0, wait_limit=0, stall_test=0,
                 fft_row_warps=0, batch_resident=0) -> rf_options:
    o = rf_options()
    o.tol, o.max_iter = float(tol), int(max_iter)
    o.green, o.ref_medium = GREEN[green], REF[ref]
    o.precision, o.check_every = PRECISION[precision], int(check_every)
    o.transform = TRANSFORM[transform]
    o.fft_rows, o.fft_cols = int(fft_rows), int(fft_cols)
    o.fft_fuse, o.fft_fuse_kx = int(fft_fuse), int(fft_fuse_kx)
    o.fft_row_blocks = int(fft_row_blocks)
    o.wait_limit, o.stall_test = int(wait_limit), int(stall_test)
    o.fft_row_warps = int(fft_row_warps)
    o.batch_resident = int(batch_resident)
    return o


def rf_pattern_adapted(phase_map, inclusion_phase, k_target, stream=None):
    pm = np.ascontiguousarray(phase_map, dtype=np.uint8)
    g = make_grid(pm.shape)
    cap = int(k_target) + 1
    out = np.zeros((cap, 3), np.int32)
    K = C.c_int64(0)
    _check(lib.rf_pattern_adapted(C.byref(g), _ptr(pm), int(inclusion_phase), int(k_target),
                                  _ptr(out), cap, C.byref(K), stream), allow_nc=False)
    return out[:K.value].copy()


def rf_pattern_adapted_noalloc(phase_map, inclusion_phase, k_target, stream=None):
    """Allocation-free variant (grids of at most 65536 voxels); see include/rf.h."""
    pm = np.ascontiguousarray(phase_map, dtype=np.uint8)
    g = make_grid(pm.shape)
    cap = int(k_target) + 1
    out = np.zeros((cap, 3), np.int32)
    K = C.c_int64(0)
    _check(lib.rf_pattern_adapted_noalloc(C.byref(g), _ptr(pm), int(inclusion_phase),
                                          int(k_target), _ptr(out), cap, C.byref(K), stream),
           allow_nc=False)
    return out[:K.value].copy()


def rf_pattern_radial(shape, k_target, stream=None):
    g = make_grid(shape)
    cap = int(k_target) + 1
    out = np.zeros((cap, 3), np.int32)
    K = C.c_int64(0)
    _check(lib.rf_pattern_radial(C.byref(g), int(k_target), _ptr(out), cap, C.byref(K), stream),
           allow_nc=False)
    return out[:K.value].copy()


class Solver:
    """One solver context (rf_create ... rf_destroy)."""

    def __init__(self, phase_map, phases, pattern=None, stream=None, **opts):
        self.pm = np.ascontiguousarray(phase_map, dtype=np.uint8)
        self.shape = self.pm.shape
        self.N = self.pm.size
        self._grid = make_grid(self.shape)
        self._phases = make_phases(phases)
        self._opts = make_options(**opts)
        self.ctx = C.c_void_p()
        _check(lib.rf_create(C.byref(self.ctx), C.byref(self._grid), len(phases), self._phases,
                             _ptr(self.pm), C.byref(self._opts), stream), allow_nc=False)
        self.K = 0
        if pattern is not None:
            self.rf_set_pattern(pattern)

    def close(self):
        if self.ctx:
            lib.rf_destroy(self.ctx)
            self.ctx = C.c_void_p()

    __del__ = close

    def rf_set_pattern(self, pattern):
        p = np.ascontiguousarray(pattern, dtype=np.int32).reshape(-1, 3)
        _check(lib.rf_set_pattern(self.ctx, _ptr(p), len(p)), allow_nc=False)
        self.K = len(p)

    def rf_set_phase_map(self, phase_map):
        pm = np.ascontiguousarray(phase_map, dtype=np.uint8)
        _check(lib.rf_set_phase_map(self.ctx, _ptr(pm)), allow_nc=False)

    def rf_set_phase_map_device(self, dev_ptr: int):
        _check(lib.rf_set_phase_map_device(self.ctx, C.c_void_p(dev_ptr)), allow_nc=False)

    def rf_solve(self, macro, warm=None):
        m = np.ascontiguousarray(macro, dtype=np.float64)
        w = None if warm is None else np.ascontiguousarray(warm, dtype=np.float32)
        sbar = np.zeros(6)
        it = C.c_int32(0)
        res = C.c_double(0)
        code = _check(lib.rf_solve(self.ctx, _ptr(m), _ptr(w), _ptr(sbar), C.byref(it),
                                   C.byref(res)))
        return dict(sigma_bar=sbar, iters=it.value, residual=res.value,
                    converged=code == RF_OK)

    def rf_solve_path(self, path):
        p = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 6)
        n = len(p)
        sbar = np.zeros((n, 6))
        its = np.zeros(n, np.int32)
        res = np.zeros(n)
        code = _check(lib.rf_solve_path(self.ctx, n, _ptr(p), _ptr(sbar), _ptr(its), _ptr(res)))
        return dict(sigma_bar=sbar, iters=its, residuals=res, converged=code == RF_OK)

    def rf_compat(self):
        """Compatibility step (one full-set update from the last reduced solve); the fields
        of rf_get_fields become the step's. Returns the homogenised stress [6]."""
        sbar = np.zeros(6)
        _check(lib.rf_compat(self.ctx, _ptr(sbar)), allow_nc=False)
        return sbar

    def rf_stress_errors(self, ref: "Solver"):
        """(Ebar, E) of Sec. 5 between this context's fields and those of `ref`."""
        eb, e = C.c_double(0.0), C.c_double(0.0)
        _check(lib.rf_stress_errors(self.ctx, ref.ctx, C.byref(eb), C.byref(e)), allow_nc=False)
        return eb.value, e.value

    def rf_solve_mixed(self, control, target, warm=None):
        """Mixed control: control[i] = 1 prescribes the average stress target[i], 0 the strain."""
        ctl = np.ascontiguousarray(control, dtype=np.int32)
        t = np.ascontiguousarray(target, dtype=np.float64)
        w = None if warm is None else np.ascontiguousarray(warm, dtype=np.float32)
        sbar, ebar = np.zeros(6), np.zeros(6)
        it = C.c_int32(0)
        res = C.c_double(0)
        code = _check(lib.rf_solve_mixed(self.ctx, _ptr(ctl), _ptr(t), _ptr(w), _ptr(sbar),
                                         _ptr(ebar), C.byref(it), C.byref(res)))
        return dict(sigma_bar=sbar, strain_bar=ebar, iters=it.value, residual=res.value,
                    converged=code == RF_OK)

    def rf_solve_path_mixed(self, control, path):
        ctl = np.ascontiguousarray(control, dtype=np.int32)
        p = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 6)
        n = len(p)
        sbar, ebar = np.zeros((n, 6)), np.zeros((n, 6))
        its = np.zeros(n, np.int32)
        res = np.zeros(n)
        code = _check(lib.rf_solve_path_mixed(self.ctx, _ptr(ctl), n, _ptr(p), _ptr(sbar),
                                              _ptr(ebar), _ptr(its), _ptr(res)))
        return dict(sigma_bar=sbar, strain_bar=ebar, iters=its, residuals=res,
                    converged=code == RF_OK)

    def rf_law_sweep(self, eps, tau, sig=None):
        """Unfused constitutive sweep on CUDA tensors eps, tau (and sig) of shape [NC, N] float32
        (enqueued on the context's stream)."""
        _check(lib.rf_law_sweep(self.ctx, _dptr(eps), _dptr(tau), _dptr(sig)), allow_nc=False)

    def rf_reset_path(self):
        _check(lib.rf_reset_path(self.ctx), allow_nc=False)

    def rf_get_fields(self):
        eps = np.zeros((6, self.N), np.float32)
        sig = np.zeros((6, self.N), np.float32)
        alpha = np.zeros(self.N, np.float32)
        _check(lib.rf_get_fields(self.ctx, _ptr(eps), _ptr(sig), _ptr(alpha)), allow_nc=False)
        sh = self.shape
        return (eps.reshape((6,) + sh), sig.reshape((6,) + sh), alpha.reshape(sh))

    def rf_get_reduced_strain(self):
        out = np.zeros((self.K, 6, 2), np.float32)
        _check(lib.rf_get_reduced_strain(self.ctx, _ptr(out)), allow_nc=False)
        return out

    def rf_get_state(self) -> bytes:
        n = C.c_size_t(0)
        _check(lib.rf_get_state(self.ctx, None, C.byref(n)), allow_nc=False)
        buf = np.zeros(n.value, np.uint8)
        _check(lib.rf_get_state(self.ctx, _ptr(buf), C.byref(n)), allow_nc=False)
        return buf.tobytes()

    def rf_set_state(self, state: bytes):
        buf = np.frombuffer(state, np.uint8).copy()
        _check(lib.rf_set_state(self.ctx, _ptr(buf), len(buf)), allow_nc=False)

    def rf_set_tracing(self, on=True):
        _check(lib.rf_set_tracing(self.ctx, int(bool(on))), allow_nc=False)

    def rf_reset_stage_times(self):
        _check(lib.rf_reset_stage_times(self.ctx), allow_nc=False)

    def rf_get_stage_times(self) -> dict:
        ms = np.zeros(8)
        n = np.zeros(8, np.int64)
        _check(lib.rf_get_stage_times(self.ctx, _ptr(ms), _ptr(n)), allow_nc=False)
        return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(STAGES)}

    def rf_get_info(self) -> dict:
        i = rf_info()
        _check(lib.rf_get_info(self.ctx, C.byref(i)), allow_nc=False)
        return {k: getattr(i, k) for k, _ in rf_info._fields_}


class BatchSolver:
    """Many independent 2D RVEs solved together (rf_batch_create ... rf_batch_destroy)."""

    def __init__(self, phase_maps, phases, patterns, stream=None, **opts):
        self.n = len(phase_maps)
        self.pms = [np.ascontiguousarray(p, dtype=np.uint8) for p in phase_maps]
        self.pats = [np.ascontiguousarray(p, dtype=np.int32).reshape(-1, 3) for p in patterns]
        self.K = [len(p) for p in self.pats]
        grids = (rf_grid * self.n)()
        for i, pm in enumerate(self.pms):
            g = make_grid(pm.shape)
            grids[i] = g
        self._grids = grids
        pm_ptrs = (C.c_void_p * self.n)(*[p.ctypes.data for p in self.pms])
        pat_ptrs = (C.c_void_p * self.n)(*[p.ctypes.data for p in self.pats])
        Ks = np.ascontiguousarray(self.K, dtype=np.int64)
        self._phases = make_phases(phases)
        self._opts = make_options(**opts)
        self.b = C.c_void_p()
        _check(lib.rf_batch_create(C.byref(self.b), self.n, grids, C.cast(pm_ptrs, C.c_void_p),
                                   len(phases), self._phases, C.cast(pat_ptrs, C.c_void_p),
                                   _ptr(Ks), C.byref(self._opts), stream), allow_nc=False)

    def close(self):
        if self.b:
            lib.rf_batch_destroy(self.b)
            self.b = C.c_void_p()

    __del__ = close

    def rf_batch_solve(self, macro, warm=None):
        m = np.ascontiguousarray(macro, dtype=np.float64).reshape(self.n, 6)
        sbar = np.zeros((self.n, 6))
        its = np.zeros(self.n, np.int32)
        res = np.zeros(self.n)
        st = np.zeros(self.n, np.int32)
        wp = None
        keep = None
        if warm is not None:
            keep = [None if w is None else np.ascontiguousarray(w, dtype=np.float32) for w in warm]
            arr = (C.c_void_p * self.n)(*[None if w is None else w.ctypes.data for w in keep])
            wp = C.cast(arr, C.c_void_p)
        code = _check(lib.rf_batch_solve(self.b, _ptr(m), wp, _ptr(sbar), _ptr(its), _ptr(res),
                                         _ptr(st)))
        del keep
        return dict(sigma_bar=sbar, iters=its, residuals=res, status=st, converged=code == RF_OK)

    def rf_batch_info(self) -> dict:
        """kernel_launches, rows_per_item for the size classes (largest side <= 64, 96, 128,
        192, larger), persistent grid size."""
        n = C.c_int64(0)
        r = np.zeros(5, np.int32)
        g = C.c_int32(0)
        _check(lib.rf_batch_info(self.b, C.byref(n), _ptr(r), C.byref(g)), allow_nc=False)
        m = C.c_int32(0)
        _check(lib.rf_batch_mode(self.b, C.byref(m)), allow_nc=False)
        return dict(kernel_launches=n.value, rows_per_item=[int(x) for x in r], grid=g.value,
                    resident=bool(m.value))


    # --- learned warm start hooks (include/rf_mlp.h); device buffers are torch CUDA tensors
    def rf_batch_slots(self):
        """(total slot count, offsets [n_rve + 1] int64 numpy)."""
        n = C.c_int64(0)
        off = np.zeros(self.n + 1, np.int64)
        _check(lib.rf_batch_slots(self.b, C.byref(n), _ptr(off)), allow_nc=False)
        return n.value, off

    def rf_batch_descriptors(self, inclusion_phase=1, rve_base=0):
        """(descriptors x [n_rve, 48], slot table [slots, 8] float32 view of rf_slot)."""
        import torch
        ns, _ = self.rf_batch_slots()
        x = torch.empty((self.n, 48), dtype=torch.float32, device="cuda")
        st = torch.empty((max(ns, 1), SLOT_FLOATS), dtype=torch.float32, device="cuda")
        _check(lib.rf_batch_descriptors(self.b, inclusion_phase, rve_base, _dptr(x), _dptr(st)),
               allow_nc=False)
        return x, st[:ns]

    def rf_batch_reduced_strain(self):
        import torch
        ns, _ = self.rf_batch_slots()
        c = torch.empty((max(ns, 1), 3, 2), dtype=torch.float32, device="cuda")
        _check(lib.rf_batch_reduced_strain(self.b, _dptr(c)), allow_nc=False)
        return c[:ns]

    def rf_batch_solve_warm(self, macro, d_warm):
        m = np.ascontiguousarray(macro, dtype=np.float64).reshape(self.n, 6)
        sbar = np.zeros((self.n, 6))
        its = np.zeros(self.n, np.int32)
        res = np.zeros(self.n)
        st = np.zeros(self.n, np.int32)
        code = _check(lib.rf_batch_solve_warm(self.b, _ptr(m), _dptr(d_warm), _ptr(sbar),
                                              _ptr(its), _ptr(res), _ptr(st)))
        return dict(sigma_bar=sbar, iters=its, residuals=res, status=st, converged=code == RF_OK)


MLP_PRECISION = {"bf16": 0, "tf32": 1}
N_IN, N_BASIS, N_OUT = 48, 27, 243


class WarmStartNet:
    """The warm-start network of include/rf_mlp.h (rf_mlp_create ... rf_mlp_destroy).

    Device inputs and outputs are torch CUDA tensors (float32 / float64 / int64 as documented
    in the header; slot tables as float32 [n, 8] views of rf_slot); parameters and gradients
    cross as flat float32 numpy arrays."""

    def __init__(self, n_hidden=512, max_batch=4096, stream=None):
        """stream: a torch.cuda.Stream; default torch's current stream, or a new stream when the
        current one is the legacy default stream. Tensors the network reads must be produced in
        order on this stream (make them inside `with torch.cuda.stream(net.stream)` and give
        BatchSolver the handle net.stream.cuda_stream)."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
            if stream.cuda_stream == 0:   # the legacy default stream: use a stream of our own
                stream = torch.cuda.Stream()
        self.stream = stream
        self.net = C.c_void_p()
        _check(lib.rf_mlp_create(C.byref(self.net), n_hidden, max_batch, _stream_handle(stream)),
               allow_nc=False)
        self.dims = self.rf_mlp_get_dims()

    def close(self):
        if self.net:
            lib.rf_mlp_destroy(self.net)
            self.net = C.c_void_p()

    __del__ = close

    def rf_mlp_get_dims(self) -> dict:
        d = rf_mlp_dims()
        _check(lib.rf_mlp_get_dims(self.net, C.byref(d)), allow_nc=False)
        return {k: getattr(d, k) for k, _ in rf_mlp_dims._fields_}

    def shapes(self):
        H = self.dims["n_hidden"]
        return [(N_IN, H), (H,), (H, H), (H,), (H, N_OUT), (N_OUT,)]

    def rf_mlp_set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.dims["n_params"]
        _check(lib.rf_mlp_set_params(self.net, _ptr(a)), allow_nc=False)

    def rf_mlp_get_params(self):
        a = np.zeros(self.dims["n_params"], np.float32)
        _check(lib.rf_mlp_get_params(self.net, _ptr(a)), allow_nc=False)
        return a

    def rf_mlp_get_grads(self):
        a = np.zeros(self.dims["n_params"], np.float32)
        _check(lib.rf_mlp_get_grads(self.net, _ptr(a)), allow_nc=False)
        return a

    def split(self, flat):
        out, o = [], 0
        for sh in self.shapes():
            n = int(np.prod(sh))
            out.append(np.asarray(flat[o:o + n]).reshape(sh))
            o += n
        return out

    def rf_mlp_forward(self, x, precision="bf16"):
        import torch
        out = torch.empty((x.shape[0], N_OUT), dtype=torch.float32, device=x.device)
        _check(lib.rf_mlp_forward(self.net, x.shape[0], _dptr(x), _dptr(out),
                                  MLP_PRECISION[precision]), allow_nc=False)
        return out

    def rf_mlp_targets(self, macro, slots, offsets, coeffs):
        """macro [B, 6] float64, slots [n, 8], offsets [B + 1] int64, coeffs [n, 3, 2]."""
        import torch
        B = macro.shape[0]
        t = torch.empty((slots.shape[0], 6), dtype=torch.float32, device=slots.device)
        e = torch.empty((B, 3), dtype=torch.float32, device=slots.device)
        _check(lib.rf_mlp_targets(self.net, B, _dptr(macro), _dptr(slots), _dptr(offsets),
                                  _dptr(coeffs), _dptr(t), _dptr(e)), allow_nc=False)
        return t, e

    def rf_mlp_loss_grad(self, x, e, slots, offsets, t, want_loss=True):
        loss = C.c_double(0.0)
        _check(lib.rf_mlp_loss_grad(self.net, x.shape[0], _dptr(x), _dptr(e), _dptr(slots),
                                    _dptr(offsets), _dptr(t),
                                    C.byref(loss) if want_loss else None), allow_nc=False)
        return loss.value if want_loss else None

    def rf_mlp_adam(self, lr):
        _check(lib.rf_mlp_adam(self.net, C.c_float(lr)), allow_nc=False)

    def rf_mlp_train_step(self, x, e, slots, offsets, t, lr, want_loss=False):
        loss = C.c_double(0.0)
        _check(lib.rf_mlp_train_step(self.net, x.shape[0], _dptr(x), _dptr(e), _dptr(slots),
                                     _dptr(offsets), _dptr(t), C.c_float(lr),
                                     C.byref(loss) if want_loss else None), allow_nc=False)
        return loss.value if want_loss else None

    def rf_mlp_predict_warm(self, x, macro, slots, offsets):
        import torch
        out = torch.empty((max(slots.shape[0], 1), 3, 2), dtype=torch.float32, device=x.device)
        _check(lib.rf_mlp_predict_warm(self.net, x.shape[0], _dptr(x), _dptr(macro),
                                       _dptr(slots), _dptr(offsets), _dptr(out)), allow_nc=False)
        return out[:slots.shape[0]]

    def rf_mlp_launches(self) -> int:
        n = C.c_int64(0)
        _check(lib.rf_mlp_launches(self.net, C.byref(n)), allow_nc=False)
        return n.value
