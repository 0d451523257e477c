"""Reduced-frequency Lippmann-Schwinger solver for GB300 (sm_103a).

The solver (Sec. 4's reduced fixed-point scheme with the geometrically adapted sampling
pattern of Sec. 4.2) lives in librf.so behind the C ABI declared in include/rf.h; `rf` is the
Python binding. Import `paper_2103_10203_gb300.rf` explicitly: it loads the CUDA library and
fails if it is missing.
"""

__all__ = ["rf"]
