"""Pins of the moving-window oracle (oracle/window_oracle.py) against what the construction
fixes, independent of the oracle's own blending code where possible:

* one window is the global fit (the whole domain, every centre): the blended surface equals
  oracle.fit's surface;
* the weights are a partition of unity: their unnormalised sum is 1 everywhere (smooth steps
  s(t) + s(1 - t) = 1 across each overlap band), for several window layouts and overlaps,
  including none;
* membership against a plain loop over the items (extended boxes grown by the margin, the
  domain's sides open);
* data generated from known weights are reproduced at the data points when no centre within
  R of a data box's inner edge carries weight: then every window's points see, among its own
  centres, all the weighted centres within R of them, so each local least-squares problem has
  a zero residual (solved by SVD least squares with no centre removed);
* the blended surface approaches the global fit as the overlap grows, and as the margin
  grows;
* a window's system with the default margin R is about as well conditioned as the global
  one on clustered terrain (the reason for the reading)."""
import numpy as np
import pytest

import datagen as dg
import oracle as O
from oracle import window_oracle as W


def _franke(seed, N=6000, M=600):
    return dg.config_franke(seed=seed, N=N, M=M)


def test_single_window_is_the_global_fit():
    pb = _franke(71)
    fits = W.fit_windows(pb.points, pb.h, pb.centres, pb.R, pb.bbox, 1, 1, 0.05, pb.R)
    c_ref, _ = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    ci, c = fits[0]
    np.testing.assert_array_equal(ci, np.arange(pb.M))
    g = W.evaluate_windows_grid(fits, pb.centres, pb.R, pb.bbox, 1, 1, 0.05, pb.kernel, 41)
    g_ref = O.evaluate_grid(c_ref, pb.centres, pb.R, pb.kernel, 41)
    assert np.abs(g - g_ref).max() <= 1e-14 * np.abs(g_ref).max()


@pytest.mark.parametrize("wx,wy,d", [(2, 2, 0.05), (3, 2, 0.1), (4, 4, 0.02), (3, 3, 0.0)])
def test_weights_partition_of_unity(wx, wy, d):
    rng = np.random.default_rng(3)
    bbox = (0.0, 0.0, 1.0, 1.0)
    Q = rng.random((20000, 2))
    Q[:50] = np.resize(np.array([[i / wx, j / wy] for i in range(wx + 1) for j in range(wy + 1)]), (50, 2))
    ex, ey = W.core_edges(0.0, 1.0, wx), W.core_edges(0.0, 1.0, wy)
    tot = np.zeros(len(Q))
    for j in range(wy):
        for i in range(wx):
            inside = W.members(Q[:, 0], ex, i, d) & W.members(Q[:, 1], ey, j, d)
            tot += W.axis_weight(Q[:, 0], ex, i, d) * W.axis_weight(Q[:, 1], ey, j, d) * inside
    np.testing.assert_allclose(tot, 1.0, rtol=0, atol=4e-15)   # a few roundings of 1


def test_membership_against_a_loop():
    rng = np.random.default_rng(4)
    P = rng.random((3000, 2)) * 1.2 - 0.1          # some items outside the box
    C = rng.random((400, 2)) * 1.2 - 0.1
    m, d, wx, wy = 0.07, 0.05, 3, 2
    got = W.windows(P, C, (0.0, 0.0, 1.0, 1.0), wx, wy, d, m)
    k = 0
    for j in range(wy):
        for i in range(wx):
            lo_x = -np.inf if i == 0 else i / wx - d
            hi_x = np.inf if i == wx - 1 else (i + 1) / wx + d
            lo_y = -np.inf if j == 0 else j / wy - d
            hi_y = np.inf if j == wy - 1 else (j + 1) / wy + d
            pts = [p for p in range(len(P))
                   if lo_x - m <= P[p, 0] <= hi_x + m and lo_y - m <= P[p, 1] <= hi_y + m]
            cen = [c for c in range(len(C))
                   if lo_x - m <= C[c, 0] <= hi_x + m and lo_y - m <= C[c, 1] <= hi_y + m]
            np.testing.assert_array_equal(got[k][0], pts)
            np.testing.assert_array_equal(got[k][1], cen)
            k += 1
    # every point in at least one window
    assert np.all(np.bincount(np.concatenate([g[0] for g in got]), minlength=len(P)) >= 1)


@pytest.mark.parametrize("m_in_R", [0.0, 1.0])
def test_data_from_known_weights_reproduced_at_the_points(m_in_R):
    rng = np.random.default_rng(5)
    C = dg.halton(2000)
    P = rng.random((12000, 2))
    R = dg.support_radius(2000, 20.0)
    d, m, n = 0.03, m_in_R * R, 3
    # no weight on centres within R of an inner data-box edge line (a_i - d - m, a_i + d + m)
    lines = np.array([i / n + s * (d + m) for i in range(1, n) for s in (-1.0, 1.0)])
    far = np.ones(len(C), bool)
    for ax in (0, 1):
        far &= np.abs(C[:, ax][:, None] - lines[None, :]).min(axis=1) >= R
    cstar = rng.normal(size=len(C)) * far
    assert far.sum() > 300
    h = O.evaluate(cstar, C, P, R, "w31")
    bbox = (0.0, 0.0, 1.0, 1.0)
    fits = W.fit_windows(P, h, C, R, bbox, n, n, d, m, "w31", min_support=0, method="lstsq")
    f = W.evaluate_windows(fits, C, P, R, bbox, n, n, d, "w31")
    assert np.abs(f - h).max() <= 1e-9 * np.abs(h).max()
    # with weight on every centre the windows' surfaces no longer reproduce the data
    h2 = O.evaluate(rng.normal(size=len(C)), C, P, R, "w31")
    fits2 = W.fit_windows(P, h2, C, R, bbox, n, n, d, m, "w31", min_support=0, method="lstsq")
    f2 = W.evaluate_windows(fits2, C, P, R, bbox, n, n, d, "w31")
    assert np.abs(f2 - h2).max() > 1e-6 * np.abs(h2).max()


def test_overlap_brings_the_surface_to_the_global_fit():
    pb = _franke(72, N=12000, M=1200)
    c_ref, _ = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    g_ref = O.evaluate_grid(c_ref, pb.centres, pb.R, pb.kernel, 65)
    errs = []
    for d in (0.0, 1 * pb.R, 2 * pb.R):
        fits = W.fit_windows(pb.points, pb.h, pb.centres, pb.R, pb.bbox, 3, 3, d, pb.R, pb.kernel)
        g = W.evaluate_windows_grid(fits, pb.centres, pb.R, pb.bbox, 3, 3, d, pb.kernel, 65)
        errs.append(np.abs(g - g_ref).max() / np.abs(g_ref).max())
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] <= 1e-2, errs
    merrs = []
    for m in (0.0, 1 * pb.R, 3 * pb.R):
        fits = W.fit_windows(pb.points, pb.h, pb.centres, pb.R, pb.bbox, 3, 3, pb.R, m, pb.kernel)
        g = W.evaluate_windows_grid(fits, pb.centres, pb.R, pb.bbox, 3, 3, pb.R, pb.kernel, 65)
        merrs.append(np.abs(g - g_ref).max() / np.abs(g_ref).max())
    assert merrs[0] > merrs[1] > merrs[2], merrs


def _kappa(P, h, C, R, kind):
    A = O.design_matrix(P, C, R, kind)
    B, _ = O.normal_system(A, h)
    free = ~O.pinned_mask(A, 3)
    Bd = B.toarray()[free][:, free]
    dg_ = np.sqrt(np.diag(Bd))
    ev = np.linalg.eigvalsh(Bd / dg_[:, None] / dg_[None, :])
    return float(ev[-1] / ev[0])


def test_margin_keeps_windows_as_well_conditioned_as_the_global_system():
    pb = dg.config_terrain(seed=82, N=20000, M=2000)
    k_glob = _kappa(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    wins = W.windows(pb.points, pb.centres, pb.bbox, 2, 3, 3 * pb.R, pb.R)
    k_win = max(_kappa(pb.points[pi], pb.h[pi], pb.centres[ci], pb.R, pb.kernel) for pi, ci in wins)
    assert k_win <= 10 * k_glob, (k_win, k_glob)
