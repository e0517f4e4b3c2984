"""Plain FP64 CPU oracle of the learned warm start (TEST INFRASTRUCTURE ONLY: imported by
tests, never by the product path).

The paper fits c by solving the normal equations from scratch. The warm start is an
addition: a small network predicts, from local statistics of the data around each centre,
an initial c_j for the solver. Its definitions, as the library implements them:

* radial features of centre j (32 numbers): the points x_i with r_ij = ||x_i - xi_j|| / R
  < 1 (the support of Algorithm 1) fall into 16 annuli, bin k holding
  k/16 <= r_ij < (k+1)/16. For each bin, the fraction n_jk / max(1, n_j) of the support's
  n_j points that lie in it, and their mean height divided by the system's height scale
  sigma = sqrt(mean_i h_i^2) (0 for an empty bin). r_ij is sqrt(dx*dx + dy*dy) / R, every
  operation rounded once in FP64, and the bin is floor(16 r_ij).
* the network: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with W1 64x32, W2 64x64, W3 1x64;
  the weights enter the products rounded to BF16 (round to nearest, ties to even), the
  biases and activations unrounded. Prediction c0_j = sigma * y(x_j); training target
  t_j = c_j / sigma of the solved system.
* the loss L = mean_j (y_j - t_j)^2, its gradient by back-propagation with respect to the
  weights as they enter the products (straight-through for the BF16 rounding).
* Adam (Kingma and Ba, 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Flat parameter vector (length NPARAM = 6337): W1 (row-major 64x32), b1 (64), W2 (row-major
64x64), b2 (64), W3 (64), b3 (1).
Pins: tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np

from .rbf_oracle import pairs_kdtree

__all__ = ["NBINS", "NFEAT", "HID", "NPARAM", "unpack", "bf16_round", "height_scale",
           "radial_features", "mlp_forward", "mlp_loss_grad", "adam_step"]

NBINS = 16
NFEAT = 2 * NBINS
HID = 64
NPARAM = HID * NFEAT + HID + HID * HID + HID + HID + 1


def unpack(p):
    """Views (W1, b1, W2, b2, W3, b3) of a flat parameter vector."""
    p = np.asarray(p)
    o = 0
    W1 = p[o:o + HID * NFEAT].reshape(HID, NFEAT); o += HID * NFEAT
    b1 = p[o:o + HID]; o += HID
    W2 = p[o:o + HID * HID].reshape(HID, HID); o += HID * HID
    b2 = p[o:o + HID]; o += HID
    W3 = p[o:o + HID]; o += HID
    b3 = p[o:o + 1]
    return W1, b1, W2, b2, W3, b3


def bf16_round(a):
    """FP32 values rounded to the nearest BF16 value (ties to even), returned as FP32.
    BF16 keeps the FP32 sign, exponent and the top 7 mantissa bits: add half of the dropped
    16-bit field, minus one unless the kept part is odd, then clear the dropped bits."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    keep_odd = (u >> 16) & 1
    u = (u + 0x7FFF + keep_odd) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def height_scale(h):
    h = np.asarray(h, np.float64)
    return float(np.sqrt(np.mean(h * h))) if h.size else 1.0


def radial_features(P, h, C, R, scale=None):
    """(M, 32) FP64 features of every centre (see the module docstring)."""
    P = np.asarray(P, np.float64)
    h = np.asarray(h, np.float64)
    C = np.asarray(C, np.float64)
    M = C.shape[0]
    if scale is None:
        scale = height_scale(h)
    i, j, r = pairs_kdtree(P, C, R)
    k = np.floor(NBINS * r).astype(np.int64)
    cnt = np.zeros((M, NBINS))
    hs = np.zeros((M, NBINS))
    np.add.at(cnt, (j, k), 1.0)
    np.add.at(hs, (j, k), h[i])
    n = cnt.sum(axis=1, keepdims=True)
    feat = np.zeros((M, NFEAT))
    feat[:, :NBINS] = cnt / np.maximum(n, 1.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        feat[:, NBINS:] = np.where(cnt > 0, hs / np.where(cnt > 0, cnt, 1.0), 0.0) / scale
    return feat


def _layers(params, round_weights):
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(params, np.float64))
    if round_weights:
        W1, W2, W3 = (bf16_round(w).astype(np.float64) for w in (W1, W2, W3))
    return W1, b1, W2, b2, W3, b3


def mlp_forward(params, X, round_weights=True):
    """y (n,) for feature rows X (n, 32), in FP64 with the weights as they enter the
    products (BF16-rounded unless round_weights is False)."""
    W1, b1, W2, b2, W3, b3 = _layers(params, round_weights)
    X = np.asarray(X, np.float64)
    a1 = np.maximum(X @ W1.T + b1, 0.0)
    a2 = np.maximum(a1 @ W2.T + b2, 0.0)
    return a2 @ W3 + b3[0]


def mlp_loss_grad(params, X, t, round_weights=True):
    """(L, g): L = mean (y - t)^2 and its gradient (flat, length NPARAM) with respect to the
    weights as they enter the products and the biases, by back-propagation in FP64."""
    W1, b1, W2, b2, W3, b3 = _layers(params, round_weights)
    X = np.asarray(X, np.float64)
    t = np.asarray(t, np.float64)
    n = X.shape[0]
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ W3 + b3[0]
    e = y - t
    L = float(np.mean(e * e))
    dy = 2.0 * e / n                      # dL/dy
    gW3 = a2.T @ dy
    gb3 = np.array([dy.sum()])
    dz2 = np.outer(dy, W3) * (z2 > 0)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return L, g


def adam_step(params, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (params, m, v)."""
    params = np.asarray(params, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
