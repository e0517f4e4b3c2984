"""Pins of the polynomial-reproduction oracle (oracle/poly_oracle.py, Section 3, Eq. 6-10)
against what the paper and the mathematics fix: exact reproduction of linear data, the
least-squares solution of the dense [A P] by an SVD-based library solver, the normal
equations of Eq. 10, the least-squares Pythagorean identity, the printed Table 4 errors with
the linear polynomial, and that adding columns never worsens a least-squares fit."""
import os

import numpy as np
import pytest

import datagen as dg
import oracle as O
from oracle import poly_oracle as PO


def _data(seed=0, N=400, M=40, R=0.3):
    rng = np.random.default_rng(seed)
    P = rng.random((N, 2))
    C = rng.random((M, 2))
    h = np.sin(3 * P[:, 0]) * np.cos(2 * P[:, 1]) + P[:, 1] ** 2 + 0.01 * rng.standard_normal(N)
    return P, h, C, R


@pytest.mark.parametrize("kind", ["w30", "w31", "w32", "w33"])
@pytest.mark.parametrize("box", [(0.0, 0.0, 1.0), (3.0, -2.0, 0.25)])
def test_linear_data_are_reproduced_exactly(kind, box):
    """h = a_x x + a_y y + a_0 is fitted with c = 0 and k = (a_x, a_y, a_0): the polynomial
    columns represent it exactly, and the least-squares solution is unique."""
    x0, y0, s = box
    rng = np.random.default_rng(1)
    P = rng.random((1500, 2)) * s + (x0, y0)
    C = dg.halton(150) * s + (x0, y0)
    a = np.array([0.7, -1.3, 0.4])
    h = P[:, 0] * a[0] + P[:, 1] * a[1] + a[2]
    c, k, _ = PO.fit_poly(P, h, C, 0.25 * s, kind)
    assert np.abs(c).max() <= 1e-9
    np.testing.assert_allclose(k, a, rtol=0, atol=1e-9 * max(1.0, abs(x0), abs(y0)))
    Q = rng.random((50, 2)) * s + (x0, y0)
    f = PO.evaluate_poly(c, k, C, Q, 0.25 * s, kind)
    np.testing.assert_allclose(f, Q[:, 0] * a[0] + Q[:, 1] * a[1] + a[2], rtol=0, atol=1e-9)


@pytest.mark.parametrize("method", ["cholesky", "lu", "cg", "qr"])
@pytest.mark.parametrize("kind", ["w31", "w33"])
def test_solvers_agree_with_svd_least_squares(method, kind):
    """(c, k) against numpy's SVD-based least squares of the dense [A P] on the unpinned
    columns (pinned centres must come out 0)."""
    P, h, C, R = _data(M=40, R=0.25)
    c, k, d = PO.fit_poly(P, h, C, R, kind, method=method)
    pin = d["pinned"]
    Ad = d["A"].toarray()[:, ~pin]
    sol = np.linalg.lstsq(np.hstack([Ad, PO.poly_basis(P)]), h, rcond=None)[0]
    got = np.concatenate([c[~pin], k])
    assert np.abs(got - sol).max() <= 1e-9 * np.abs(sol).max()
    assert np.all(c[pin] == 0.0)


def test_normal_equations_of_eq10_hold():
    """[A P]^T (h - A c - P k) = 0 on the unpinned columns, and the bordered matrix is
    symmetric with the blocks A^T A, A^T P, P^T P."""
    P, h, C, R = _data(seed=2, N=600, M=60, R=0.25)
    c, k, d = PO.fit_poly(P, h, C, R, "w31")
    A, Pm, pin = d["A"].toarray(), d["P"], d["pinned"]
    e = h - A @ c - Pm @ k
    g = np.concatenate([(A.T @ e)[~pin], Pm.T @ e])
    scale = np.abs(np.concatenate([A.T @ h, Pm.T @ h])).max()
    assert np.abs(g).max() <= 1e-10 * scale
    K = d["K"].toarray()
    np.testing.assert_allclose(K, K.T, rtol=0, atol=1e-12 * np.abs(K).max())
    M = A.shape[1]
    np.testing.assert_allclose(K[:M, :M], A.T @ A, rtol=0, atol=1e-12 * np.abs(K).max())
    np.testing.assert_allclose(K[:M, M:], A.T @ Pm, rtol=0, atol=1e-12 * np.abs(K).max())
    np.testing.assert_allclose(K[M:, M:], Pm.T @ Pm, rtol=0, atol=1e-12 * np.abs(K).max())


def test_least_squares_pythagoras():
    """At the least-squares solution the fit and the error are orthogonal:
    ||h||^2 = ||f||^2 + ||h - f||^2 with f = A c + P k."""
    P, h, C, R = _data(seed=3)
    c, k, d = PO.fit_poly(P, h, C, R, "w32")
    f = d["A"] @ c + d["P"] @ k
    lhs = h @ h
    rhs = f @ f + (h - f) @ (h - f)
    assert abs(lhs - rhs) <= 1e-10 * lhs


def test_polynomial_never_worsens_the_fit():
    """The fit with the polynomial minimises over a superset of columns of the fit without
    it, so its residual norm is not larger (and it is smaller for data with a trend)."""
    P, h, C, R = _data(seed=4)
    h = h + 5.0 * P[:, 0] - 2.0 * P[:, 1]
    c0, ref = O.fit(P, h, C, R, "w31")
    e0 = np.linalg.norm(h - ref["A"] @ c0)
    c, k, d = PO.fit_poly(P, h, C, R, "w31")
    e1 = np.linalg.norm(h - d["A"] @ c - d["P"] @ k)
    assert e1 < e0


def test_table4_synthetic_with_linear_polynomial(golden_dir):
    rows = [l.split() for l in open(os.path.join(golden_dir, "table4_synthetic_linear.txt"))
            if l.strip() and not l.startswith("#")]
    P = dg.halton(1089)
    h = dg.franke(P[:, 0], P[:, 1])
    C = dg.halton(81)
    for kind, alpha, mae in rows:
        R = 1.0 / float(alpha)
        c, k, _ = PO.fit_poly(P, h, C, R, kind, min_support=0, method="qr")
        got = O.error_measures(PO.evaluate_poly(c, k, C, P, R, kind), h)["mae"]
        assert abs(got - float(mae)) <= 0.15 * float(mae), (kind, got, mae)
