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


def test_support_radius_gives_k_centres_per_disc():
    # reading: pi R^2 M = K on the unit square
    for M, K in ((100_000, 30.0), (2_000_000, 30.0), (2_000, 20.0)):
        R = dg.support_radius(M, K)
        assert abs(np.pi * R * R * M - K) <= 1e-9 * K


def test_bigdata_density_varies_ten_to_one():
    """Points are uniform draws kept with probability (1 + 9 s(x)) / 10, s a value-noise field
    scaled to [0, 1] by its range: the density varies 10:1, so on a 16 x 16 grid the densest
    cell holds several times the points of the sparsest, at most about ten times (up to
    sampling noise)."""
    big = dg.config_bigdata(N=400_000, M=4_000)
    H, _, _ = np.histogram2d(big.points[:, 0], big.points[:, 1], bins=16, range=[[0, 1], [0, 1]])
    ratio = H.max() / H.min()
    assert 5.0 < ratio < 13.0, ratio
    assert big.h.std() > 0 and np.isfinite(big.h).all()


def test_tile_sizes_log_uniform_in_range():
    """N_t = round(exp(U[ln 2e3, ln 2e5])), M_t = N_t // 10, independent seeds."""
    ts = dg.tile_batch(1000, 200)
    N = np.array([t.N for t in ts])
    assert N.min() >= 2000 and N.max() <= 200000
    assert all(t.M == t.N // 10 for t in ts)
    ln = np.log(N)
    mid = 0.5 * (np.log(2e3) + np.log(2e5))
    half = 0.5 * (np.log(2e5) - np.log(2e3))
    # uniform on [mid - half, mid + half]: mean at mid, standard deviation half / sqrt(3)
    assert abs(ln.mean() - mid) < 0.25 * half
    assert abs(ln.std() - half / np.sqrt(3)) < 0.2 * half
    assert len({t.N for t in ts}) > 150
