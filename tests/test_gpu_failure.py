"""Failure detection through the C ABI, in forms that fault, trap or hang no GPU.

* Non-finite input (a NaN macroscopic strain) is rejected on the host: RF_ERR_NONFINITE.
* A finite macroscopic strain so large that the FP32 fields overflow makes the device-side
  convergence measure non-finite: the solve ends with RF_ERR_NONFINITE and the context stays
  usable.
* A bounded device-side wait that runs out: the tensor-core kernels' stall test waits on a
  barrier that nothing completes, with a short poll limit; the solve returns RF_ERR_TIMEOUT,
  the kernels release their tensor memory, and later solves in the same process still match
  the oracle.
* Divergence (RF_ERR_DIVERGED) is covered with the batched solver in test_gpu_batch.py.
"""

import numpy as np
import pytest

import oracle as O
from oracle.rf_oracle import VOIGT
from synth import centred_disc
from synth.configs import elastic_phases

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))


def vec6_field(t):
    g = t[0] if t.shape[0] == 1 else t
    return np.stack([g[..., i, j] for (i, j) in VOIGT])


def _case():
    pm = centred_disc(32, 0.3)
    return pm, elastic_phases(), O.pattern_adapted(pm, 1, 103)


def test_nan_macro_strain_is_rejected(lib):
    pm, ph, pat = _case()
    s = lib.Solver(pm, ph, pattern=pat, tol=1e-6)
    with pytest.raises(lib.RFError) as e:
        s.rf_solve(np.array([np.nan, 0, 0, 0, 0, 0]))
    assert e.value.code == -3
    with pytest.raises(lib.RFError) as e:
        s.rf_solve_path(np.array([[0.01, 0, 0, 0, 0, 0], [np.inf, 0, 0, 0, 0, 0]]))
    assert e.value.code == -3
    s.close()


@pytest.mark.parametrize("transform", ["dft", "fft"])
def test_fp32_overflow_is_reported_and_the_context_stays_usable(lib, transform):
    pm, ph, pat = _case()
    s = lib.Solver(pm, ph, pattern=pat, tol=1e-6, max_iter=50, transform=transform)
    with pytest.raises(lib.RFError) as e:
        s.rf_solve(np.array([1e37, 0, 0, 0, 0, 0]))
    assert e.value.code == -3
    macro = np.array([0.01, 0, 0, 0, 0, 0.002])
    out = s.rf_solve(macro)
    s.close()
    r = O.solve(pm, ph, macro, pat, tol=1e-6)
    assert out["converged"] and rel(out["sigma_bar"], r.sigma_bar) <= 1e-6


@pytest.mark.parametrize("prec", ["split_bf16", "split_tf32"])
def test_tensor_core_wait_timeout_is_reported(lib, prec):
    pm, ph, pat = _case()
    macro = np.array([0.01, 0, 0, 0, 0, 0.002])
    s = lib.Solver(pm, ph, pattern=pat, tol=1e-6, max_iter=20, precision=prec, stall_test=1,
                   wait_limit=64)
    with pytest.raises(lib.RFError) as e:
        s.rf_solve(macro)
    assert e.value.code == -6
    s.close()
    # tensor memory was released and the context is usable: a normal split-precision solve in
    # the same process matches the oracle at the split-mode tolerance
    s = lib.Solver(pm, ph, pattern=pat, tol=0.0, max_iter=6, precision=prec, wait_limit=1 << 20)
    out = s.rf_solve(macro)
    eps, _, _ = s.rf_get_fields()
    s.close()
    r = O.solve(pm, ph, macro, pat, tol=0.0, max_iter=6)
    assert rel(eps, vec6_field(r.eps)) <= 3e-5
    assert rel(out["sigma_bar"], r.sigma_bar) <= 3e-5


def test_wait_limit_and_stall_options_are_checked(lib):
    pm, ph, pat = _case()
    with pytest.raises(lib.RFError):
        lib.Solver(pm, ph, stall_test=1)                   # FP32 has no tensor-core waits
    with pytest.raises(lib.RFError):
        lib.Solver(pm, ph, precision="split_bf16", wait_limit=-1)
