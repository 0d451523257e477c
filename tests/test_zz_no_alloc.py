"""The allocation-free adapted-pattern entry point (for callers that cannot allocate device
memory) must return exactly what rf_pattern_adapted returns.

This file is named to be collected last, so that a run stopping at the first failure has
already run every other test. It passes alone in a fresh process and after the other tests.
"""

import ctypes as C

import numpy as np
import pytest

from synth import centred_disc, random_discs, random_spheres

pytestmark = pytest.mark.gpu


def test_noalloc_pattern_matches_allocating_entry_point_twice_in_a_row(lib):
    cases = [(random_discs(96, (6.0, 14.0), 0.4, seed=5), 461),
             (random_spheres(24, (2.0, 5.0), 0.25, seed=8), 277),
             (centred_disc(64, 0.3), 205)]
    for pm, K in cases:
        want = lib.rf_pattern_adapted(pm, 1, K)
        first = lib.rf_pattern_adapted_noalloc(pm, 1, K)
        second = lib.rf_pattern_adapted_noalloc(pm, 1, K)
        # integer index work: bit-exact
        assert np.array_equal(first, want)
        assert np.array_equal(second, want)


def test_noalloc_pattern_matches_where_amplitudes_vanish(lib):
    """Cases where many selected frequencies have a quantised amplitude of zero (their ranking
    keys lie in the top half of the key range): a map without inclusion voxels, a laminate
    once K exceeds its nonzero axis, and the full set K = N. Both entry points and the oracle
    must give the same pattern."""
    import oracle as O
    from synth import laminate
    cases = [(np.zeros((32, 48), np.uint8), 37),
             (laminate((64, 64), (20, 45)), 205),
             ((np.random.default_rng(3).random((12, 20)) < 0.3).astype(np.uint8), 240)]
    for pm, K in cases:
        want = lib.rf_pattern_adapted(pm, 1, K)
        assert np.array_equal(want, O.pattern_adapted(pm, 1, K))
        for _ in range(2):
            got = lib.rf_pattern_adapted_noalloc(pm, 1, K)
            assert len(got) >= K and np.array_equal(got, want)


def test_noalloc_rejects_grids_beyond_its_static_scratch(lib):
    pm = np.zeros((257, 256), np.uint8)          # 65792 voxels > 65536
    g = lib.make_grid(pm.shape)
    out = np.zeros((10, 3), np.int32)
    K = C.c_int64(0)
    code = lib.lib.rf_pattern_adapted_noalloc(C.byref(g), C.c_void_p(pm.ctypes.data), 1, 5,
                                              C.c_void_p(out.ctypes.data), 10, C.byref(K), None)
    assert code == -1 and b"65536" in lib.lib.rf_last_error()
