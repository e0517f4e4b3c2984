"""Oracle of the moving-window fit (the "moving window" technique the paper names as future
work, Section 7): the domain is cut into overlapping windows, each window is fitted on its own
(Section 2's least squares on the window's points and the centres whose support reaches them),
and the surface is the windows' local surfaces blended by a partition of unity.

TEST INFRASTRUCTURE ONLY (see the package docstring): plain numpy / scipy, FP64.

Definitions (the paper gives the technique's name only; these are the library's readings):

* windows: wx x wy over bbox = (x0, y0, x1, y1); the core edges along x are
  a_i = x0 + (x1 - x0) * i / wx (i = 0 .. wx), likewise along y;
* window (i, j)'s extended box: [a_i - d, a_{i+1} + d] x [b_j - d, b_{j+1} + d] (closed),
  d the overlap; a side on the boundary of bbox extends to infinity, so that items outside
  bbox belong to the edge windows;
* its data box: the extended box grown by a margin m >= 0 on its inner sides (the library's
  default m = R); its points and its centres: those in the data box. A centre at the data
  box's edge keeps at least about half of its support's points, so a window's system is
  about as well conditioned as the global one; taking the centres of a box grown by R around
  the points instead leaves centres whose support holds a sliver of the window's points
  (condition numbers up to ~1e14 on clustered terrain against ~1e5 globally);
* its fit: the least-squares weights of those points and centres (oracle.fit); the window's
  surface is used inside its extended box only;
* the surface at q: sum_w w_w(q) f_w(q) / sum_w w_w(q) over the windows whose extended box
  holds q, with w_w = rho_x(q_x) rho_y(q_y) and rho along x for window i the product of
  s((q_x - (a_i - d)) / (2 d)) (when i > 0) and s(((a_{i+1} + d) - q_x) / (2 d)) (when
  i < wx - 1), s(t) = t^2 (3 - 2 t) on [0, 1], 0 below, 1 above. Two neighbours' factors
  are s(t) and s(1 - t) across their common band of width 2 d, so the weights already sum to
  one; with d = 0 the factors are steps (q_x >= a_i, q_x < a_{i+1}) and each node belongs to
  one window.
"""
from __future__ import annotations

import numpy as np

from . import rbf_oracle as O


def core_edges(lo, hi, n):
    """a_i = lo + (hi - lo) * i / n, i = 0 .. n, in the library's operation order."""
    return np.array([lo + (hi - lo) * i / n for i in range(n + 1)], np.float64)


def extended_range(edges, i, d):
    """Closed interval of window index i along one axis, infinite on the domain's sides."""
    n = len(edges) - 1
    lo = -np.inf if i == 0 else edges[i] - d
    hi = np.inf if i == n - 1 else edges[i + 1] + d
    return lo, hi


def members(v, edges, i, d, grow=0.0):
    """Mask of the coordinates v inside window i's extended interval grown by `grow`."""
    lo, hi = extended_range(edges, i, d)
    if np.isfinite(lo):
        lo = lo - grow
    if np.isfinite(hi):
        hi = hi + grow
    return (v >= lo) & (v <= hi)


def smooth_step(t):
    t = np.clip(t, 0.0, 1.0)
    return t * t * (3.0 - 2.0 * t)


def axis_weight(v, edges, i, d):
    """rho along one axis for window i at coordinates v."""
    n = len(edges) - 1
    w = np.ones_like(np.asarray(v, np.float64))
    if d > 0.0:
        if i > 0:
            w = w * smooth_step((v - (edges[i] - d)) / (2.0 * d))
        if i < n - 1:
            w = w * smooth_step(((edges[i + 1] + d) - v) / (2.0 * d))
    else:
        if i > 0:
            w = w * (v >= edges[i])
        if i < n - 1:
            w = w * (v < edges[i + 1])
    return w


def windows(P, C, bbox, wx, wy, d, m):
    """Per window (i, j) in row-major order (j slow): (point indices, centre indices) of the
    items in its data box (extended box grown by the margin m)."""
    ex = core_edges(bbox[0], bbox[2], wx)
    ey = core_edges(bbox[1], bbox[3], wy)
    out = []
    for j in range(wy):
        for i in range(wx):
            pm = members(P[:, 0], ex, i, d, m) & members(P[:, 1], ey, j, d, m)
            cm = members(C[:, 0], ex, i, d, m) & members(C[:, 1], ey, j, d, m)
            out.append((np.nonzero(pm)[0], np.nonzero(cm)[0]))
    return out


def fit_windows(P, h, C, R, bbox, wx, wy, d, m, kind="w31", min_support=3, method="cholesky"):
    """Each window's weights: a list of (centre indices, c) in window order."""
    P = np.asarray(P, np.float64)
    C = np.asarray(C, np.float64)
    h = np.asarray(h, np.float64)
    res = []
    for pi, ci in windows(P, C, bbox, wx, wy, d, m):
        if ci.size == 0:
            res.append((ci, np.zeros(0)))
            continue
        if pi.size == 0:
            res.append((ci, np.zeros(ci.size)))
            continue
        if method == "lstsq":
            # least squares by SVD (numpy's lstsq): the minimum-norm solution also when a
            # centre of the halo has no point of the window in its support
            A = O.design_matrix(P[pi], C[ci], R, kind).toarray()
            pin = O.pinned_mask(A, min_support) if min_support > 0 else np.zeros(ci.size, bool)
            c = np.zeros(ci.size)
            keep = np.nonzero(~pin)[0]
            c[keep] = np.linalg.lstsq(A[:, keep], h[pi], rcond=None)[0]
        else:
            c, _ = O.fit(P[pi], h[pi], C[ci], R, kind, method=method, min_support=min_support)
        res.append((ci, c))
    return res


def evaluate_windows(fits, C, Q, R, bbox, wx, wy, d, kind="w31"):
    """The blended surface at query points Q (K x 2)."""
    Q = np.asarray(Q, np.float64)
    C = np.asarray(C, np.float64)
    ex = core_edges(bbox[0], bbox[2], wx)
    ey = core_edges(bbox[1], bbox[3], wy)
    num = np.zeros(Q.shape[0])
    den = np.zeros(Q.shape[0])
    k = 0
    for j in range(wy):
        for i in range(wx):
            ci, c = fits[k]
            k += 1
            inside = members(Q[:, 0], ex, i, d) & members(Q[:, 1], ey, j, d)
            w = axis_weight(Q[:, 0], ex, i, d) * axis_weight(Q[:, 1], ey, j, d) * inside
            sel = np.nonzero(w > 0.0)[0]
            if sel.size == 0:
                continue
            f = O.evaluate(c, C[ci], Q[sel], R, kind) if ci.size else np.zeros(sel.size)
            num[sel] += w[sel] * f
            den[sel] += w[sel]
    return num / den


def evaluate_windows_grid(fits, C, R, bbox, wx, wy, d, kind, n, box=None):
    """The blended surface on the node-centred n x n grid over box (bbox by default)."""
    x0, y0, x1, y1 = bbox if box is None else box
    X, Y = np.meshgrid(np.linspace(x0, x1, n), np.linspace(y0, y1, n))
    Q = np.stack([X.ravel(), Y.ravel()], 1)
    return evaluate_windows(fits, C, Q, R, bbox, wx, wy, d, kind).reshape(n, n)
