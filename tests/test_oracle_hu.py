"""Pins of the oracle's CT HU -> impedance pre-pass: breakpoints map to
their values, a two-point table is an affine map, the ends clamp, and the
map is the textbook linear interpolation numpy provides."""
import numpy as np
import pytest

import oracle

TABLE_HU = [-1000.0, -100.0, 0.0, 40.0, 1000.0, 3000.0]
TABLE_Z = [0.0004, 1.38, 1.48, 1.62, 6.0, 7.8]


def test_breakpoints_and_clamping():
    hu = np.array([-1024, -1000, -100, 0, 40, 1000, 3000, 3071], np.int16)
    z = oracle.hu_to_z(hu, TABLE_HU, TABLE_Z)
    np.testing.assert_array_equal(z, [0.0004, 0.0004, 1.38, 1.48, 1.62, 6.0, 7.8, 7.8])


def test_two_point_table_is_affine():
    hu = np.arange(-500, 501, 7, dtype=np.int16)
    z = oracle.hu_to_z(hu, [-500.0, 500.0], [1.0, 3.0])
    np.testing.assert_allclose(z, 2.0 + hu / 500.0, rtol=0, atol=1e-15)


def test_matches_numpy_interp():
    rng = np.random.default_rng(2)
    hu = rng.integers(-1100, 3200, size=5000).astype(np.int16)
    np.testing.assert_allclose(oracle.hu_to_z(hu, TABLE_HU, TABLE_Z), np.interp(hu, TABLE_HU, TABLE_Z),
                               rtol=1e-15, atol=1e-15)


def test_rejects_unsorted_table():
    with pytest.raises(ValueError):
        oracle.hu_to_z(np.zeros(3, np.int16), [0.0, 0.0], [1.0, 2.0])
