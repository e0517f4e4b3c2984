"""Checks of the seeded input generators (shapes, ranges, determinism, Halton values)."""
import numpy as np

import datagen as dg


def test_halton_first_values():
    H = dg.halton(4)
    np.testing.assert_allclose(H[:, 0], [1 / 2, 1 / 4, 3 / 4, 1 / 8])
    np.testing.assert_allclose(H[:, 1], [1 / 3, 2 / 3, 1 / 9, 4 / 9])


def test_franke_known_maximum_region():
    # the largest Franke bump sits near (2/9, 2/9)
    v = dg.franke(np.array([2 / 9]), np.array([2 / 9]))[0]
    assert 1.0 < v < 1.3


def test_configs_deterministic_and_in_box():
    a = dg.config_franke(N=500, M=50)
    b = dg.config_franke(N=500, M=50)
    assert np.array_equal(a.points, b.points) and np.array_equal(a.h, b.h)
    assert a.points.min() >= 0 and a.points.max() < 1
    t = dg.config_terrain(N=5000, M=500)
    assert t.points.shape == (5000, 2) and t.points.min() >= 0 and t.points.max() < 1
    assert abs(t.R - dg.support_radius(500, 30)) == 0.0
    tl = dg.tile(1000)
    assert 2000 <= tl.N <= 200000 and tl.M == tl.N // 10
    big = dg.config_bigdata(N=20000, M=2000)
    assert big.points.shape == (20000, 2) and big.kernel == "w32"
