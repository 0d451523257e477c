"""CPU-side checks of the C ABI: the library loads, exports every declared symbol, and rejects
invalid arguments before touching the GPU."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                  if f.endswith(".h"))
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(rf_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def rf():
    from paper_2103_10203_gb300.build import build
    build()
    from paper_2103_10203_gb300 import rf as mod
    return mod


def test_library_exports_every_declared_symbol(rf):
    names = declared_symbols()
    assert len(names) >= 16
    for n in names:
        assert hasattr(rf.lib, n), n
    assert sorted(rf.EXPORTED) == names


def test_struct_layouts_match_header(rf, tmp_path):
    """sizeof/offsetof of every ABI struct as the C compiler lays them out from rf.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"rf_grid": rf.rf_grid, "rf_phase": rf.rf_phase, "rf_options": rf.rf_options,
               "rf_info": rf.rf_info, "rf_mlp_dims": rf.rf_mlp_dims, "rf_slot": rf.rf_slot}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rf_mlp.h"', "int main(void){"]
    for name, py in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in py._fields_:
            cf = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {cf}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    want = dict(line.split() for line in out.strip().splitlines())
    for name, py in structs.items():
        assert int(want[name]) == C.sizeof(py), name
        for fname, _ in py._fields_:
            assert int(want[f"{name}.{fname}"]) == getattr(py, fname).offset, (name, fname)


def _create(rf, pm, phases, **kw):
    g = rf.make_grid(pm.shape) if "grid" not in kw else kw.pop("grid")
    opts = rf.make_options(**kw)
    ctx = C.c_void_p()
    ph = rf.make_phases(phases)
    code = rf.lib.rf_create(C.byref(ctx), C.byref(g), len(phases), ph,
                            C.c_void_p(pm.ctypes.data), C.byref(opts), None)
    return code, ctx


def test_invalid_arguments_are_rejected_on_the_host(rf):
    from synth import phase_table
    pm = np.zeros((8, 8), np.uint8)
    good = phase_table([(1.0, 1.0, 0, 0, 0)])
    bad_grid = rf.rf_grid()
    bad_grid.dim = 4
    code, _ = _create(rf, pm, good, grid=bad_grid)
    assert code == -1 and b"dim" in rf.lib.rf_last_error()
    g = rf.make_grid(pm.shape)
    g.n[2] = 2
    code, _ = _create(rf, pm, good, grid=g)
    assert code == -1 and b"Nz" in rf.lib.rf_last_error()
    code, _ = _create(rf, pm, phase_table([(1.0, -1.0, 0, 0, 0)]))
    assert code == -1 and b"mu > 0" in rf.lib.rf_last_error()
    code, _ = _create(rf, pm, phase_table([(1.0, 1.0, 0.0, 0.1, 1)]))
    assert code == -1 and b"sigma_y0" in rf.lib.rf_last_error()
    code, _ = _create(rf, pm, good, max_iter=0)
    assert code == -1
    assert rf.lib.rf_create(None, None, 0, None, None, None, None) == -1
    assert rf.lib.rf_destroy(None) == 0


def test_pattern_arguments_rejected_on_the_host(rf):
    g = rf.make_grid((8, 8))
    out = np.zeros((4, 3), np.int32)
    K = C.c_int64(0)
    pm = np.zeros((8, 8), np.uint8)
    code = rf.lib.rf_pattern_adapted(C.byref(g), C.c_void_p(pm.ctypes.data), 1, 0,
                                     C.c_void_p(out.ctypes.data), 4, C.byref(K), None)
    assert code == -1
    g3 = rf.make_grid((4, 8, 8))
    code = rf.lib.rf_pattern_radial(C.byref(g3), 5, C.c_void_p(out.ctypes.data), 4, C.byref(K),
                                    None)
    assert code == -1 and b"2D" in rf.lib.rf_last_error()


def test_network_and_batch_hooks_reject_invalid_arguments_on_the_host(rf):
    net = C.c_void_p()
    assert rf.lib.rf_mlp_create(C.byref(net), 20, 8, None) == -1      # hidden % 16 != 0
    assert b"n_hidden" in rf.lib.rf_last_error()
    assert rf.lib.rf_mlp_create(C.byref(net), 32, 0, None) == -1
    assert rf.lib.rf_mlp_create(None, 32, 8, None) == -1
    n = C.c_int64(0)
    assert rf.lib.rf_batch_slots(None, C.byref(n), None) == -1
    assert rf.lib.rf_batch_descriptors(None, 1, 0, None, None) == -1
    assert rf.lib.rf_batch_reduced_strain(None, None) == -1
    assert rf.lib.rf_batch_solve_warm(None, None, None, None, None, None, None) == -1
    assert rf.lib.rf_mlp_destroy(None) == 0


def test_non_finite_moduli_are_rejected_on_the_host(rf):
    """NaN or infinite moduli give RF_ERR_NONFINITE before any device work (single context and
    batch)."""
    from synth import phase_table
    pm = np.zeros((8, 8), np.uint8)
    for bad in ([(np.nan, 1.0, 0, 0, 0)], [(1.0, np.inf, 0, 0, 0)], [(1.0, 1.0, np.nan, 1.0, 1)]):
        code, ctx = _create(rf, pm, phase_table(bad))
        assert code == -3 and not ctx.value
        assert b"finite" in rf.lib.rf_last_error()
    g = (rf.rf_grid * 1)(rf.make_grid(pm.shape))
    pat = np.zeros((1, 3), np.int32)
    pm_ptrs = (C.c_void_p * 1)(pm.ctypes.data)
    pat_ptrs = (C.c_void_p * 1)(pat.ctypes.data)
    Ks = np.ones(1, np.int64)
    opts = rf.make_options()
    b = C.c_void_p()
    ph = rf.make_phases(phase_table([(np.nan, 1.0, 0, 0, 0)]))
    code = rf.lib.rf_batch_create(C.byref(b), 1, g, C.cast(pm_ptrs, C.c_void_p), 1, ph,
                                  C.cast(pat_ptrs, C.c_void_p), C.c_void_p(Ks.ctypes.data),
                                  C.byref(opts), None)
    assert code == -3 and not b.value
