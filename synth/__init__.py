"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the bench.

This package holds no arithmetic of the reduced-frequency method itself: it only draws
microstructures (phase maps), macroscopic strains and material constants. The paper's own
geometries exist only as figures (Sec. 5), so every workload here is a synthetic stand-in
shaped like the paper's examples: one centred circular/spherical inclusion (Sec. 5.1, 5.3) and
composites with several circular inclusions (Sec. 5.2).
"""

from .microstructure import (  # noqa: F401
    centred_annulus,
    centred_disc,
    centred_ellipse,
    centred_square,
    centred_sphere,
    laminate,
    random_discs,
    random_spheres,
    random_macro_strain,
)
from .materials import lame, phase_table  # noqa: F401
from .configs import CONFIGS, make_config  # noqa: F401
