"""The seeded input generators (synth) for the full-size workloads: shapes and
sizes as stated, and the 1-D scaling series as nested prefixes of one line of
cubes. No method arithmetic is involved; these pin the inputs the GPU tests
and bench.py use."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("name,n", [("cube32", 98_304), ("slab256", 393_216), ("cube48", 331_776),
                                    ("cube64v", 786_432), ("array4096", 786_432)])
def test_workload_sizes(name, n):
    v = synth.workload(name).voxels
    assert 3 * v.centres.shape[0] == n
    assert np.all(np.isfinite(v.centres)) and np.all(np.real(v.eps_r) >= 1.0)


def test_cube_array_series_is_nested():
    """arrayNNN: NNN cubes of 4^3 voxels on the x axis, pitch 0.5, eps_r 2.54;
    every member is a prefix of the longest one, and the generic name gives
    the same 4096-cube line as the named workload."""
    full = synth.workload("array4096").voxels
    for c in (512, 1024, 2048, 4096):
        w = synth.workload(f"array{c}")
        v = w.voxels
        assert v.centres.shape[0] == 64 * c
        np.testing.assert_array_equal(v.centres, full.centres[:64 * c])
        assert np.all(v.eps_r == 2.54)
        assert (w.n_min, w.eta, w.eps) == (96, 1.0, 1e-4)
    # the line grows along x only, one cube every 0.5
    x = full.centres[:, 0].reshape(4096, 64)
    assert np.allclose(np.diff(x.min(axis=1)), 0.5)
    assert np.ptp(full.centres[:, 1]) == np.ptp(full.centres[:64, 1])
