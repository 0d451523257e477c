"""FP64 CPU oracle of the reduced-frequency Moulinec-Suquet scheme.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call, link or execute
anything in this package: only the tests, the smoke check of the entry module and the
CPU-baseline leg of the benchmark use it. It shares no code with the CUDA library.

The oracle is plain and slow on purpose: it follows the paper's reduced fixed-point scheme
(Sec. 4, steps a-d) in the paper's order, in float64, with numpy's FFT as the transform
step (the paper's own implementation restricts a full FFT to the reduced set, Sec. 4).

Parity pins (tests/test_oracle_*.py, marked "not gpu") tie every function here to something
other than itself: brute-force DFT sums, closed-form Green operators, projector identities,
homogeneous/Voigt/laminate closed forms, Hashin-Shtrikman bounds, the J2 uniaxial closed
form, a brute-force Galerkin solve and Dirichlet-kernel amplitudes for patterns.
The fixed radial sampling pattern (Sec. 4.1) is the one function whose definition the paper
gives only as a figure: "parity unpinned" for `pattern_radial` beyond its structural checks.
"""

from .rf_oracle import (  # noqa: F401
    forward_reduced,
    inverse_reduced,
    isotropic_stiffness,
    SolveResult,
    compat,
    errors,
    full_pattern,
    green_operator,
    law,
    pattern_adapted,
    pattern_radial,
    reference_medium,
    solve,
    solve_path,
    tensor_to_vec6,
    vec6_to_tensor,
    wave_vector,
)
