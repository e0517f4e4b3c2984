"""Plain, slow, FP64 CPU oracle for CS-RBF least-squares approximation
(Majdisova & Skala, "Big Geo Data Surface Approximation using Radial Basis
Functions: A Comparative Study").

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.

What it computes, step by step, in the paper's notation:

* phi      -- Wendland CS-RBFs of Table 2 with the cut-off of Eq. 18, written in
              r = ||x - xi|| / R (R = 1/alpha).  phi_{3,2} is not in Table 2; it
              is the catalogue form (1-r)^6 (35 r^2 + 18 r + 3) divided by 3 so
              that phi(0) = 1 like the others.
* A        -- the N x M matrix A_ij = phi(||x_i - xi_j|| / R) of Eq. 4-5, built
              as COO triplets {i, j, phi} exactly as Algorithm 1 emits them: a
              kd-tree range query finds every pair with ||x_i - xi_j|| < R.
* B, b     -- the normal system B = A^T A (Eq. 11-12), b = A^T h (Section 2);
              ``normal_system_blocked`` computes only the upper-triangle blocks
              B_kl = A_{*,k}^T A_{*,l}, l >= k (Eq. 13-14) and mirrors them.
* pinning  -- a centre whose support disc holds fewer than ``min_support`` data
              points is removed from the system and its weight set to 0 (the
              paper is silent on empty supports; this is the reading used by
              both implementations).
* c        -- the least-squares weights, solving B c = b on the remaining
              centres: dense Cholesky, dense QR least squares of A (the textbook
              route for small N), sparse LU, or Jacobi-preconditioned CG.
* f        -- the approximant f(x) = sum_j c_j phi(||x - xi_j|| / R) (Eq. 3).

Parity pins for every function live in ``tests/test_oracle.py``.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg
from scipy.spatial import cKDTree

__all__ = [
    "phi", "pairs_bruteforce", "pairs_kdtree", "design_matrix", "normal_system",
    "normal_system_blocked", "support_counts", "pinned_mask", "solve_normal",
    "solve_lstsq_qr", "pcg", "evaluate", "evaluate_grid", "fit", "normal_residual",
    "coo_spmv", "rel_err", "error_measures", "SampledOracle",
]

_KINDS = ("w30", "w31", "w32", "w33")


# ----------------------------------------------------------------------------
# basis functions (Table 2, Eq. 18)
# ----------------------------------------------------------------------------

def phi(r, kind: str = "w31"):
    """Wendland phi_{3,s}(r) for r = ||x - xi|| / R >= 0; zero for r >= 1 (Eq. 18)."""
    r = np.asarray(r, dtype=np.float64)
    inside = r < 1.0
    t = np.where(inside, 1.0 - r, 0.0)                       # (1 - r)_+
    if kind == "w30":
        v = t ** 2
    elif kind == "w31":
        v = t ** 4 * (4.0 * r + 1.0)
    elif kind == "w32":
        v = t ** 6 * (35.0 * r * r + 18.0 * r + 3.0) / 3.0
    elif kind == "w33":
        v = t ** 8 * (32.0 * r ** 3 + 25.0 * r * r + 8.0 * r + 1.0)
    else:
        raise ValueError(f"unknown kernel {kind!r}")
    return np.where(inside, v, 0.0)


def _dist_over_R(P, C, i, j, R):
    """r = sqrt(dx^2 + dy^2) / R for the pairs (i, j)."""
    dx = P[i, 0] - C[j, 0]
    dy = P[i, 1] - C[j, 1]
    return np.sqrt(dx * dx + dy * dy) / R


# ----------------------------------------------------------------------------
# neighbour search (Algorithm 1, line 3)
# ----------------------------------------------------------------------------

def pairs_bruteforce(P, C, R, chunk: int = 2048):
    """All (i, j, r) with r = ||x_i - xi_j|| / R < 1, by checking every pair."""
    P = np.asarray(P, np.float64)
    C = np.asarray(C, np.float64)
    I, J, Rr = [], [], []
    for i0 in range(0, P.shape[0], chunk):
        i1 = min(P.shape[0], i0 + chunk)
        dx = P[i0:i1, 0, None] - C[None, :, 0]
        dy = P[i0:i1, 1, None] - C[None, :, 1]
        r = np.sqrt(dx * dx + dy * dy) / R
        ii, jj = np.nonzero(r < 1.0)
        I.append(ii + i0)
        J.append(jj)
        Rr.append(r[ii, jj])
    if not I:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0)
    return np.concatenate(I).astype(np.int64), np.concatenate(J).astype(np.int64), np.concatenate(Rr)


def pairs_kdtree(P, C, R):
    """All (i, j, r) with r < 1, via a kd-tree range query over the given points
    (Algorithm 1: build the tree once, query it for every reference point).  The
    tree returns a slightly widened candidate set; membership is then decided with
    the same r < 1 test as ``pairs_bruteforce``."""
    P = np.asarray(P, np.float64)
    C = np.asarray(C, np.float64)
    if P.shape[0] == 0 or C.shape[0] == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0)
    tp = cKDTree(P)
    tc = cKDTree(C)
    S = tp.sparse_distance_matrix(tc, R * (1.0 + 1e-9), output_type="coo_matrix")
    i = S.row.astype(np.int64)
    j = S.col.astype(np.int64)
    r = _dist_over_R(P, C, i, j, R)
    keep = r < 1.0
    i, j, r = i[keep], j[keep], r[keep]
    order = np.lexsort((j, i))
    return i[order], j[order], r[order]


# ----------------------------------------------------------------------------
# the overdetermined system and the normal equations
# ----------------------------------------------------------------------------

def design_matrix(P, C, R, kind="w31", search="kdtree"):
    """A (N x M, scipy COO) with A_ij = phi(||x_i - xi_j|| / R) (Eq. 4-5, Algorithm 1)."""
    f = pairs_kdtree if search == "kdtree" else pairs_bruteforce
    i, j, r = f(P, C, R)
    return scipy.sparse.coo_matrix((phi(r, kind), (i, j)), shape=(len(P), len(C)))


def normal_system(A, h):
    """B = A^T A (Eq. 11-12) and b = A^T h, in FP64."""
    A = scipy.sparse.csr_matrix(A)
    B = (A.T @ A).tocsr()
    b = A.T @ np.asarray(h, np.float64)
    return B, np.asarray(b).ravel()


def normal_system_blocked(A, h, MB: int):
    """B from its upper-triangle blocks only: B_kl = (A_{*,k})^T A_{*,l} for l >= k
    (Eq. 13-14), the lower triangle filled by symmetry.  Returned dense."""
    A = scipy.sparse.csc_matrix(A)
    M = A.shape[1]
    nb = -(-M // MB)
    B = np.zeros((M, M))
    for k in range(nb):
        k0, k1 = k * MB, min(M, (k + 1) * MB)
        Ak = A[:, k0:k1]
        for l in range(k, nb):
            l0, l1 = l * MB, min(M, (l + 1) * MB)
            Bkl = (Ak.T @ A[:, l0:l1]).toarray()
            B[k0:k1, l0:l1] = Bkl
            if l != k:
                B[l0:l1, k0:k1] = Bkl.T
    b = A.T @ np.asarray(h, np.float64)
    return B, np.asarray(b).ravel()


def support_counts(A):
    """Number of data points strictly inside each centre's support disc (column nnz of A)."""
    A = scipy.sparse.csc_matrix(A)
    return np.diff(A.indptr).astype(np.int64)


def pinned_mask(A, min_support: int = 3):
    """Centres with fewer than min_support points in their support: removed, c_j = 0."""
    return support_counts(A) < min_support


# ----------------------------------------------------------------------------
# solvers for B c = b
# ----------------------------------------------------------------------------

def pcg(B, b, tol=1e-14, maxit=100_000, x0=None):
    """Jacobi-preconditioned conjugate gradients in FP64 on the SPD system B x = b.
    Stops when ||b - B x||_2 <= tol ||b||_2.  Returns (x, iterations, rel_residual)."""
    B = scipy.sparse.csr_matrix(B)
    d = B.diagonal().copy()
    dinv = 1.0 / d
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    r = b - B @ x
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, 0.0
    z = dinv * r
    p = z.copy()
    rz = r @ z
    it = 0
    rel = np.linalg.norm(r) / nb
    while rel > tol and it < maxit:
        q = B @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        rel = np.linalg.norm(r) / nb
    return x, it, rel


def solve_normal(B, b, pinned=None, method="cholesky", tol=1e-14, maxit=100_000):
    """Solve B c = b on the unpinned centres; pinned centres get c_j = 0.
    method: 'cholesky' (dense LL^T), 'lu' (sparse LU), 'cg' (Jacobi-PCG FP64)."""
    M = B.shape[0]
    free = np.ones(M, bool) if pinned is None else ~np.asarray(pinned, bool)
    idx = np.nonzero(free)[0]
    c = np.zeros(M)
    if idx.size == 0:
        return c
    Bs = scipy.sparse.csr_matrix(B)[idx][:, idx]
    bs = b[idx]
    if method == "cholesky":
        cf = scipy.linalg.cho_factor(Bs.toarray(), lower=True)
        c[idx] = scipy.linalg.cho_solve(cf, bs)
    elif method == "lu":
        c[idx] = scipy.sparse.linalg.spsolve(Bs.tocsc(), bs)
    elif method == "cg":
        c[idx] = pcg(Bs, bs, tol=tol, maxit=maxit)[0]
    else:
        raise ValueError(method)
    return c


def solve_lstsq_qr(A, h, pinned=None):
    """min ||A c - h||_2 by Householder QR of the dense A (Section 2, 'least squares')."""
    A = scipy.sparse.csr_matrix(A)
    M = A.shape[1]
    free = np.ones(M, bool) if pinned is None else ~np.asarray(pinned, bool)
    idx = np.nonzero(free)[0]
    Ad = A[:, idx].toarray()
    Q, Rm = scipy.linalg.qr(Ad, mode="economic")
    c = np.zeros(M)
    c[idx] = scipy.linalg.solve_triangular(Rm, Q.T @ np.asarray(h, np.float64))
    return c


# ----------------------------------------------------------------------------
# evaluation (Eq. 3)
# ----------------------------------------------------------------------------

def evaluate(c, C, Q, R, kind="w31"):
    """f(q) = sum_j c_j phi(||q - xi_j|| / R) at query points Q (K x 2)."""
    Q = np.asarray(Q, np.float64)
    i, j, r = pairs_kdtree(Q, C, R)
    f = np.zeros(Q.shape[0])
    np.add.at(f, i, np.asarray(c)[j] * phi(r, kind))
    return f


def evaluate_grid(c, C, R, kind, n, bbox=(0.0, 0.0, 1.0, 1.0)):
    """f on the node-centred n x n grid over bbox, returned (n, n) with f[iy, ix]."""
    x0, y0, x1, y1 = bbox
    gx = np.linspace(x0, x1, n)
    gy = np.linspace(y0, y1, n)
    X, Y = np.meshgrid(gx, gy)
    return evaluate(c, C, np.stack([X.ravel(), Y.ravel()], 1), R, kind).reshape(n, n)


# ----------------------------------------------------------------------------
# the whole fit, residuals, measures
# ----------------------------------------------------------------------------

def fit(P, h, C, R, kind="w31", method=None, min_support=3, tol=1e-14, search="kdtree"):
    """Least-squares CS-RBF weights c (original centre order) and diagnostics."""
    A = design_matrix(P, C, R, kind, search)
    B, b = normal_system(A, h)
    pin = pinned_mask(A, min_support)
    if method is None:
        method = "cholesky" if B.shape[0] <= 4000 else "cg"
    c = solve_normal(B, b, pin, method, tol=tol)
    return c, dict(A=A, B=B, b=b, pinned=pin, method=method)


def normal_residual(A, h, c):
    """A^T (h - A c) in FP64 (the normal-equation residual)."""
    A = scipy.sparse.csr_matrix(A)
    return np.asarray(A.T @ (np.asarray(h, np.float64) - A @ np.asarray(c, np.float64))).ravel()


def coo_spmv(row, col, data, x, nrows):
    """y = Q x with Q in coordinate format, entry by entry as in Section 4."""
    y = np.zeros(nrows, dtype=np.result_type(np.asarray(data), np.asarray(x)))
    for k in range(len(data)):
        y[row[k]] = y[row[k]] + data[k] * x[col[k]]
    return y


def rel_err(u, ref):
    """max_i |u_i - ref_i| / max_i |ref_i| (norm-wise max relative error)."""
    u = np.asarray(u, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.max(np.abs(ref)) if ref.size else 0.0
    num = np.max(np.abs(u - ref)) if ref.size else 0.0
    return float(num / den) if den > 0 else float(num)


def error_measures(f_approx, f_true):
    """Table 4 style measures: mean absolute error, variance and standard deviation of the
    error, and mean |error| relative to the height range."""
    e = np.asarray(f_approx) - np.asarray(f_true)
    rng = float(np.max(f_true) - np.min(f_true))
    return dict(mae=float(np.mean(np.abs(e))), var=float(np.var(e)), std=float(np.std(e)),
                mre_range=float(np.mean(np.abs(e)) / rng) if rng > 0 else float("nan"))


# ----------------------------------------------------------------------------
# sampled quantities at sizes where the whole system is too large for the CPU
# ----------------------------------------------------------------------------

class SampledOracle:
    """Entries of A, B = A^T A, b = A^T h, the normal residual and f, computed one by one
    from their definitions (Eq. 3-5, 11-12) with kd-tree range queries."""

    def __init__(self, P, h, C, R, kind="w31"):
        self.P = np.asarray(P, np.float64)
        self.h = np.asarray(h, np.float64)
        self.C = np.asarray(C, np.float64)
        self.R = float(R)
        self.kind = kind
        self.tp = cKDTree(self.P)
        self.tc = cKDTree(self.C)

    def _near(self, tree, X, q):
        idx = np.asarray(tree.query_ball_point(q, self.R * (1.0 + 1e-9)), dtype=np.int64)
        if idx.size == 0:
            return idx, np.zeros(0)
        dx = X[idx, 0] - q[0]
        dy = X[idx, 1] - q[1]
        r = np.sqrt(dx * dx + dy * dy) / self.R
        keep = r < 1.0
        return idx[keep], r[keep]

    def row(self, i):
        """Nonzeros of row i of A: (centre indices, values)."""
        j, r = self._near(self.tc, self.C, self.P[i])
        return j, phi(r, self.kind)

    def column(self, j):
        """Nonzeros of column j of A: (point indices, values)."""
        i, r = self._near(self.tp, self.P, self.C[j])
        return i, phi(r, self.kind)

    def B_entry(self, j, k):
        ij, vj = self.column(j)
        ik, vk = self.column(k)
        common, aj, ak = np.intersect1d(ij, ik, assume_unique=True, return_indices=True)
        return float(np.sum(vj[aj] * vk[ak]))

    def b_entry(self, j):
        i, v = self.column(j)
        return float(np.sum(v * self.h[i]))

    def support(self, j):
        return int(self.column(j)[0].size)

    def normal_residual(self, c, j):
        """(A^T (h - A c))_j."""
        i, v = self.column(j)
        e = np.empty(i.size)
        for t, ii in enumerate(i):
            jj, vv = self.row(ii)
            e[t] = self.h[ii] - np.sum(vv * c[jj])
        return float(np.sum(v * e))

    def f(self, c, q):
        """f(q) = sum_j c_j phi(||q - xi_j|| / R)."""
        j, r = self._near(self.tc, self.C, np.asarray(q, np.float64))
        return float(np.sum(np.asarray(c)[j] * phi(r, self.kind)))
