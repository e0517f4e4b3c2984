"""Pins for the CPU FP64 oracle: each check compares the oracle with something
other than itself -- the Wendland functions' defining integral recursion, the
worked COO example and the Table 4 errors printed in the paper, brute force on
tiny inputs, library least-squares routines, and invariants (symmetry, positive
semi-definiteness, block invariance of Eq. 13, exact interpolation, the
Pythagorean identity of least squares)."""
import math
import os

import numpy as np
import pytest
import scipy.sparse
from numpy.polynomial import Polynomial as Pn

import datagen as dg
import oracle as O


# ----------------------------------------------------------------------------
# basis functions
# ----------------------------------------------------------------------------

def _wendland_by_definition(k: int, d: int = 3):
    """phi_{d,k} from its definition: (1-r)^l with l = floor(d/2)+k+1, then k applications
    of (I f)(r) = int_r^1 t f(t) dt, normalised to 1 at r = 0.  Exact polynomial algebra."""
    l = d // 2 + k + 1
    f = Pn([1.0, -1.0]) ** l
    t = Pn([0.0, 1.0])
    for _ in range(k):
        F = (t * f).integ()
        f = F(1.0) - F
    return f / f(0.0)


@pytest.mark.parametrize("kind,k", [("w30", 0), ("w31", 1), ("w32", 2), ("w33", 3)])
def test_phi_matches_wendland_recursion(kind, k):
    r = np.linspace(0.0, 0.999, 1001)
    ref = _wendland_by_definition(k)(r)
    # the monomial-form reference loses ~1e-13 to cancellation near r = 1; phi(0) = 1
    np.testing.assert_allclose(O.phi(r, kind), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kind", dg.KERNELS)
def test_phi_support_and_origin(kind):
    assert O.phi(0.0, kind) == 1.0
    assert np.all(O.phi(np.array([1.0, 1.0 + 1e-12, 1.5, 10.0]), kind) == 0.0)
    r = np.linspace(0, 1, 2001)
    assert np.all(O.phi(r, kind) >= 0.0)
    assert np.all(np.diff(O.phi(r, kind)) <= 1e-15)       # non-increasing


@pytest.mark.parametrize("kind,s", [("w30", 0), ("w31", 1), ("w32", 2), ("w33", 3)])
def test_phi_order_of_contact_at_edge(kind, s):
    """phi_{3,s} is C^{2s}: it meets zero at r = 1 to order exactly 2s + 2, so
    phi(1 - e) / e^(2s+2) tends to a finite nonzero limit; for s >= 1 phi'(0) = 0."""
    q = 2 * s + 2
    vals = [O.phi(1.0 - e, kind) / e ** q for e in (1e-3, 1e-4, 1e-5)]
    assert vals[-1] > 0.0
    assert abs(vals[1] - vals[2]) < 1e-2 * vals[2]
    assert abs(vals[0] - vals[2]) < 1e-1 * vals[2]
    if s >= 1:
        d0 = (O.phi(1e-6, kind) - O.phi(0.0, kind)) / 1e-6
        assert abs(d0) < 1e-4


@pytest.mark.parametrize("kind", dg.KERNELS)
def test_phi_positive_definite_2d(kind):
    """Table 2's functions are positive definite in up to 3 dimensions: the interpolation
    matrix on distinct 2-D points is SPD."""
    rng = np.random.default_rng(5)
    X = rng.random((150, 2))
    D = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    Phi = O.phi(D / 0.4, kind)
    assert np.allclose(Phi, Phi.T)
    assert np.linalg.eigvalsh(Phi).min() > 0.0


# ----------------------------------------------------------------------------
# neighbour search and the COO format
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_kdtree_pairs_equal_bruteforce(seed):
    rng = np.random.default_rng(seed)
    P = rng.random((3000, 2))
    C = rng.random((400, 2))
    R = 0.07
    a = O.pairs_kdtree(P, C, R)
    b = O.pairs_bruteforce(P, C, R)
    ka = set(zip(a[0].tolist(), a[1].tolist()))
    kb = set(zip(b[0].tolist(), b[1].tolist()))
    assert ka == kb and len(ka) > 1000


def _read_coo_golden(golden_dir):
    Q, arr = [], {}
    with open(os.path.join(golden_dir, "coo_example_Q.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            if tok[0] == "Q":
                Q.append([float(x) for x in tok[1:]])
            else:
                arr[tok[0]] = np.array([int(x) for x in tok[1:]])
    return np.array(Q), arr


def test_coo_worked_example(golden_dir):
    Q, arr = _read_coo_golden(golden_dir)
    y1 = O.coo_spmv(arr["row"], arr["col"], arr["data"], np.ones(5), 5)
    np.testing.assert_array_equal(y1, Q @ np.ones(5))
    np.testing.assert_array_equal(y1, [7, 18, 12, 10, 5])
    x = np.array([3, -1, 4, 1, -5], dtype=np.float64)
    np.testing.assert_array_equal(O.coo_spmv(arr["row"], arr["col"], arr["data"], x, 5), Q @ x)


# ----------------------------------------------------------------------------
# the normal system
# ----------------------------------------------------------------------------

def _tiny(seed=3, N=70, M=16, R=0.35, kind="w31"):
    rng = np.random.default_rng(seed)
    return rng.random((N, 2)), rng.standard_normal(N), rng.random((M, 2)), R, kind


def test_normal_matrix_equals_bruteforce_gram():
    P, h, C, R, kind = _tiny()
    Ad = np.zeros((len(P), len(C)))
    for i in range(len(P)):
        for j in range(len(C)):
            d = math.hypot(P[i, 0] - C[j, 0], P[i, 1] - C[j, 1])
            Ad[i, j] = O.phi(d / R, kind)
    A = O.design_matrix(P, C, R, kind)
    np.testing.assert_allclose(A.toarray(), Ad, rtol=0, atol=1e-15)
    B, b = O.normal_system(A, h)
    np.testing.assert_allclose(B.toarray(), Ad.T @ Ad, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(b, Ad.T @ h, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("kind", dg.KERNELS)
def test_normal_matrix_symmetric_psd(kind):
    pb = dg.config_small(7, 4000, 600, K=20.0, kernel=kind)
    A = O.design_matrix(pb.points, pb.centres, pb.R, kind)
    B, _ = O.normal_system(A, pb.h)
    Bd = B.toarray()
    assert np.array_equal(Bd, Bd.T)
    ev = np.linalg.eigvalsh(Bd)
    assert ev.min() >= -1e-12 * ev.max()


@pytest.mark.parametrize("MB", [1, 7, 40, 600])
def test_block_partition_invariance(MB):
    pb = dg.config_small(11, 3000, 600)
    A = O.design_matrix(pb.points, pb.centres, pb.R, pb.kernel)
    B, b = O.normal_system(A, pb.h)
    Bb, bb = O.normal_system_blocked(A, pb.h, MB)
    np.testing.assert_allclose(Bb, B.toarray(), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(bb, b, rtol=1e-13)


# ----------------------------------------------------------------------------
# the least-squares solution
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("kind", dg.KERNELS)
def test_solvers_agree_with_library_lstsq(kind):
    pb = dg.config_small(13, 400, 60, K=12.0, kernel=kind)
    A = O.design_matrix(pb.points, pb.centres, pb.R, kind)
    B, b = O.normal_system(A, pb.h)
    pin = O.pinned_mask(A)
    free = ~pin
    c_np = np.zeros(pb.M)
    c_np[free] = np.linalg.lstsq(A.toarray()[:, free], pb.h, rcond=None)[0]
    c_qr = O.solve_lstsq_qr(A, pb.h, pin)
    c_ch = O.solve_normal(B, b, pin, "cholesky")
    c_cg = O.solve_normal(B, b, pin, "cg", tol=1e-15)
    c_lu = O.solve_normal(B, b, pin, "lu")
    for c in (c_qr, c_ch, c_cg, c_lu):
        assert O.rel_err(c, c_np) < 1e-9


def test_least_squares_pythagoras_and_normal_residual():
    pb = dg.config_franke(N=3000, M=300)
    c, info = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    A = info["A"]
    res = O.normal_residual(A, pb.h, c)
    assert np.max(np.abs(res)) <= 1e-10 * np.max(np.abs(info["b"]))
    e0 = A @ c - pb.h
    rng = np.random.default_rng(0)
    for _ in range(5):
        d = rng.standard_normal(pb.M)
        e1 = A @ (c + d) - pb.h
        Ad = A @ d
        assert abs((e1 @ e1 - e0 @ e0) - Ad @ Ad) <= 1e-8 * (Ad @ Ad)


@pytest.mark.parametrize("kind", dg.KERNELS)
def test_interpolation_reproduces_data(kind):
    """M = N with xi = x: A is the SPD interpolation matrix (Eq. 1-2), so h is reproduced."""
    rng = np.random.default_rng(21)
    X = rng.random((300, 2))
    h = dg.franke(X[:, 0], X[:, 1])
    c, info = O.fit(X, h, X, 0.15, kind, min_support=1)
    assert np.max(np.abs(info["A"] @ c - h)) <= 1e-10 * np.max(np.abs(h))


def test_pinned_centre_gets_zero_weight():
    pb = dg.config_small(17, 2000, 200)
    C = pb.centres.copy()
    C[5] = (0.5, 0.5)
    P = pb.points[np.hypot(pb.points[:, 0] - 0.5, pb.points[:, 1] - 0.5) > 2 * pb.R]
    h = pb.h[np.hypot(pb.points[:, 0] - 0.5, pb.points[:, 1] - 0.5) > 2 * pb.R]
    c, info = O.fit(P, h, C, pb.R, pb.kernel)
    assert info["pinned"][5] and c[5] == 0.0
    keep = ~info["pinned"]
    A = info["A"].tocsc()[:, keep]
    c_ref = np.linalg.lstsq(A.toarray(), h, rcond=None)[0]
    assert O.rel_err(c[keep], c_ref) < 1e-9


# ----------------------------------------------------------------------------
# evaluation (Eq. 3) and the paper's own numbers
# ----------------------------------------------------------------------------

def test_evaluate_equals_bruteforce_sum():
    rng = np.random.default_rng(4)
    C = rng.random((50, 2))
    c = rng.standard_normal(50)
    Q = rng.random((40, 2)) * 1.2 - 0.1
    R = 0.3
    ref = np.array([sum(c[j] * O.phi(math.hypot(q[0] - C[j, 0], q[1] - C[j, 1]) / R, "w33")
                        for j in range(50)) for q in Q])
    np.testing.assert_allclose(O.evaluate(c, C, Q, R, "w33"), ref, rtol=1e-13, atol=1e-15)
    F = O.evaluate_grid(c, C, R, "w33", 7)
    g = np.linspace(0, 1, 7)
    np.testing.assert_allclose(F[2, 5], O.evaluate(c, C, np.array([[g[5], g[2]]]), R, "w33")[0])


def test_table4_synthetic_mean_absolute_error(golden_dir):
    rows = [l.split() for l in open(os.path.join(golden_dir, "table4_synthetic.txt"))
            if l.strip() and not l.startswith("#")]
    P = dg.halton(1089)
    h = dg.franke(P[:, 0], P[:, 1])
    C = dg.halton(81)
    for kind, alpha, mae in rows:
        A = O.design_matrix(P, C, 1.0 / float(alpha), kind)
        c = O.solve_lstsq_qr(A, h)
        got = O.error_measures(A @ c, h)["mae"]
        assert abs(got - float(mae)) <= 0.15 * float(mae), (kind, got, mae)


def test_rel_err_definition():
    assert O.rel_err([1.0, 2.0], [1.0, 4.0]) == 0.5
    assert O.rel_err([0.0], [0.0]) == 0.0


def test_sampled_oracle_matches_full_system():
    pb = dg.config_terrain(N=6000, M=600)
    A = O.design_matrix(pb.points, pb.centres, pb.R, pb.kernel)
    B, b = O.normal_system(A, pb.h)
    c, _ = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    cpert = c + 1e-3 * np.random.default_rng(1).standard_normal(pb.M)
    res = O.normal_residual(A, pb.h, cpert)
    so = O.SampledOracle(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    Bd = B.toarray()
    sup = O.support_counts(A)
    F = A @ cpert
    for j in [0, 7, 123, 599]:
        assert abs(so.b_entry(j) - b[j]) <= 1e-12 * max(1.0, abs(b[j]))
        assert so.support(j) == sup[j]
        assert abs(so.normal_residual(cpert, j) - res[j]) <= 1e-10 * np.abs(res).max()
        for k in [j, (j + 1) % 600, (j + 37) % 600]:
            assert abs(so.B_entry(j, k) - Bd[j, k]) <= 1e-13 * Bd.max()
    for i in [0, 5, 4000]:
        assert abs(so.f(cpert, pb.points[i]) - F[i]) <= 1e-12 * np.abs(F).max()
