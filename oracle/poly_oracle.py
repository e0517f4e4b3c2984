"""Plain FP64 CPU oracle of the RBF approximation with linear polynomial reproduction
(TEST INFRASTRUCTURE ONLY: imported by tests, never by the product path).

Section 3 (Eq. 6-10): the approximant gains a linear polynomial,
    f(x) = sum_j c_j phi(||x - xi_j|| / R) + a_x x + a_y y + a_0,
and the fit minimises ||A c + P k - h||_2 over c and k = (a_x, a_y, a_0), where A is the
design matrix of Eq. 4-5 and row i of P is (x_i, y_i, 1) (Eq. 8-9). Its normal equations are
the bordered system of Eq. 10,
    [ A^T A   A^T P ] [c]   [A^T h]
    [ P^T A   P^T P ] [k] = [P^T h],
symmetric positive definite whenever [A P] has full column rank. This is least squares, not
interpolation: there are no orthogonality constraint rows, so the system is solved as one SPD
system. As in the fit without the polynomial, centres with fewer than min_support points
strictly inside their support leave the system (c_j = 0); the three polynomial unknowns are
always kept.
Pins: tests/test_oracle_poly.py.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

from .rbf_oracle import design_matrix, evaluate, pcg, pinned_mask

__all__ = ["poly_basis", "bordered_system", "fit_poly", "evaluate_poly"]

NPOLY = 3


def poly_basis(P):
    """P (N x 3): row i is (x_i, y_i, 1) (Eq. 9)."""
    P = np.asarray(P, np.float64)
    return np.column_stack([P[:, 0], P[:, 1], np.ones(len(P))])


def bordered_system(A, Pm, h):
    """The matrix and right-hand side of Eq. 10 (scipy CSR, FP64): unknowns c (M) then k (3)."""
    A = scipy.sparse.csr_matrix(A)
    Pm = np.asarray(Pm, np.float64)
    h = np.asarray(h, np.float64)
    AtA = (A.T @ A).tocsr()
    AtP = np.asarray(A.T @ Pm)                 # M x 3
    PtP = Pm.T @ Pm                            # 3 x 3
    K = scipy.sparse.bmat([[AtA, scipy.sparse.csr_matrix(AtP)],
                           [scipy.sparse.csr_matrix(AtP.T), scipy.sparse.csr_matrix(PtP)]],
                          format="csr")
    rhs = np.concatenate([np.asarray(A.T @ h).ravel(), Pm.T @ h])
    return K, rhs


def fit_poly(P, h, C, R, kind="w31", min_support=3, method=None, tol=1e-14):
    """(c, k, diagnostics): the least-squares weights c (original centre order, pinned centres
    0) and polynomial coefficients k = (a_x, a_y, a_0). method: 'cholesky' (dense, default for
    M <= 4000), 'lu' (sparse LU), 'cg' (Jacobi-preconditioned CG) on Eq. 10, or 'qr'
    (Householder QR of the dense [A P], for small systems whose Eq. 10 matrix is too
    ill-conditioned to factor, e.g. supports wider than the domain)."""
    A = design_matrix(P, C, R, kind)
    Pm = poly_basis(P)
    K, rhs = bordered_system(A, Pm, h)
    M = A.shape[1]
    pin = pinned_mask(A, min_support)
    keep = np.concatenate([np.nonzero(~pin)[0], M + np.arange(NPOLY)])
    Ks = K[keep][:, keep]
    rs = rhs[keep]
    if method is None:
        method = "cholesky" if keep.size <= 4000 else "lu"
    if method == "qr":
        Ad = np.hstack([scipy.sparse.csr_matrix(A)[:, keep[:-NPOLY]].toarray(), Pm])
        Q, Rm = scipy.linalg.qr(Ad, mode="economic")
        xs = scipy.linalg.solve_triangular(Rm, Q.T @ np.asarray(h, np.float64))
    elif method == "cholesky":
        cf = scipy.linalg.cho_factor(Ks.toarray(), lower=True)
        xs = scipy.linalg.cho_solve(cf, rs)
    elif method == "lu":
        xs = scipy.sparse.linalg.spsolve(Ks.tocsc(), rs)
    elif method == "cg":
        xs, _, _ = pcg(Ks, rs, tol=tol)
    else:
        raise ValueError(method)
    x = np.zeros(M + NPOLY)
    x[keep] = xs
    return x[:M], x[M:], dict(A=A, P=Pm, K=K, rhs=rhs, pinned=pin, method=method)


def evaluate_poly(c, k, C, Q, R, kind="w31"):
    """f(q) = sum_j c_j phi(||q - xi_j|| / R) + a_x q_x + a_y q_y + a_0 (Eq. 6-7)."""
    Q = np.asarray(Q, np.float64)
    k = np.asarray(k, np.float64)
    return evaluate(c, C, Q, R, kind) + Q[:, 0] * k[0] + Q[:, 1] * k[1] + k[2]
