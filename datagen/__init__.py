"""Seeded synthetic inputs for the CS-RBF least-squares surface fit.

This module is shared by the CPU oracle's tests and by the GPU path's tests and
benchmark.  It produces input arrays only -- point sets, heights, centre sets,
the support radius and the evaluation grid -- and holds none of the method's
arithmetic (no basis function, no normal equations, no solver).

Workloads (the paper's LiDAR sets are not available, so these stand in for
them; Section 6 of the paper uses Halton points with Franke heights for its
synthetic experiment):

* ``config_franke``     N uniform points in [0,1]^2, Franke heights (Eq. 17)
                        plus N(0, 0.01^2) noise, M Halton centres.
* ``config_terrain``    N points from a 64-Gaussian mixture over a 20 % uniform
                        floor, heights from 200 Gaussian bumps plus 6-octave
                        value noise, M Halton centres.  The floor puts about
                        2K points in every support disc even between the
                        clusters (with N/M = 10), so the least-squares problem
                        stays overdetermined everywhere; without it the
                        Halton centres outnumber the points 2:1 between the
                        clusters and A^T A is numerically singular.
* ``config_bigdata``    N points with 10:1 density variation (rejection
                        sampling against 3-octave value noise), heights from an
                        8-octave value-noise terrain, M Halton centres.
* ``tile``              one tile of the batched workload: N log-uniform in
                        [2e3, 2e5], M = N // 10, Halton centres with a per-tile
                        index offset, heights s*Franke(affine(x)) + 0.3*noise +
                        N(0, 0.01^2).

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64).  The
support radius follows "about K centres per support disc": pi R^2 M = K on the
unit square.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem", "halton", "franke", "value_noise", "support_radius", "grid_nodes",
    "config_franke", "config_terrain", "config_bigdata", "tile", "tile_batch",
    "config_small", "KERNELS", "mlp_init", "MLP_NPARAM",
]

KERNELS = ("w30", "w31", "w32", "w33")


@dataclass
class Problem:
    """One fitting problem: data points, heights, centres and the support radius."""

    points: np.ndarray          # (N, 2) float64
    h: np.ndarray               # (N,)  float64
    centres: np.ndarray         # (M, 2) float64
    R: float                    # support radius (1/alpha)
    kernel: str = "w31"         # Wendland function name, one of KERNELS
    bbox: tuple = (0.0, 0.0, 1.0, 1.0)   # (x0, y0, x1, y1) containing all points and centres
    eval_n: int = 256           # output grid is eval_n x eval_n nodes over bbox
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.points.shape[0])

    @property
    def M(self) -> int:
        return int(self.centres.shape[0])


# ----------------------------------------------------------------------------
# point sets
# ----------------------------------------------------------------------------

def _radical_inverse(idx: np.ndarray, base: int) -> np.ndarray:
    """Van der Corput radical inverse of integer indices in the given base."""
    idx = idx.astype(np.int64).copy()
    out = np.zeros(idx.shape, dtype=np.float64)
    f = 1.0 / base
    while np.any(idx > 0):
        out += f * (idx % base)
        idx //= base
        f /= base
    return out


def halton(n: int, start: int = 1, bases=(2, 3)) -> np.ndarray:
    """Halton points with indices start .. start+n-1 (index 0 is the origin and is skipped
    by the default start=1); no scrambling, no leaping."""
    idx = np.arange(start, start + n, dtype=np.int64)
    return np.stack([_radical_inverse(idx, b) for b in bases], axis=1)


# ----------------------------------------------------------------------------
# height functions
# ----------------------------------------------------------------------------

def franke(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Franke's test function (Eq. 17 of the paper)."""
    f1 = 0.75 * np.exp(-((9 * x - 2) ** 2) / 4.0 - ((9 * y - 2) ** 2) / 4.0)
    f2 = 0.75 * np.exp(-((9 * x + 1) ** 2) / 49.0 - ((9 * y + 1) ** 2) / 10.0)
    f3 = 0.50 * np.exp(-((9 * x - 7) ** 2) / 4.0 - ((9 * y - 3) ** 2) / 4.0)
    f4 = 0.20 * np.exp(-((9 * x - 4) ** 2) - ((9 * y - 7) ** 2))
    return f1 + f2 + f3 - f4


def _fade(t: np.ndarray) -> np.ndarray:
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def value_noise(x, y, rng: np.random.Generator, octaves: int, base: int = 4,
                lacunarity: float = 2.0, persistence: float = 0.5) -> np.ndarray:
    """Fractal value noise on [0,1]^2: per octave a lattice of uniform [-1,1] values
    (drawn from ``rng``), quintic-fade bilinear interpolation, amplitudes persistence^o.
    The result is normalised by the sum of amplitudes, so it lies in [-1, 1]."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out = np.zeros(np.broadcast(x, y).shape, dtype=np.float64)
    amp, total = 1.0, 0.0
    for o in range(octaves):
        L = int(round(base * lacunarity ** o))
        lat = rng.uniform(-1.0, 1.0, size=(L + 1, L + 1))
        gx = np.clip(x, 0.0, 1.0) * L
        gy = np.clip(y, 0.0, 1.0) * L
        ix = np.minimum(gx.astype(np.int64), L - 1)
        iy = np.minimum(gy.astype(np.int64), L - 1)
        tx = _fade(gx - ix)
        ty = _fade(gy - iy)
        v00 = lat[ix, iy]
        v10 = lat[ix + 1, iy]
        v01 = lat[ix, iy + 1]
        v11 = lat[ix + 1, iy + 1]
        a = v00 + tx * (v10 - v00)
        b = v01 + tx * (v11 - v01)
        out += amp * (a + ty * (b - a))
        total += amp
        amp *= persistence
    return out / total


def _noise_fn(rng: np.random.Generator, octaves: int, base: int, persistence: float = 0.5):
    """Freeze the lattices of one value-noise field so it can be sampled repeatedly."""
    seed = int(rng.integers(0, 2**63 - 1))

    def f(x, y):
        return value_noise(x, y, np.random.default_rng(seed), octaves, base=base,
                           persistence=persistence)
    return f


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def support_radius(M: int, K: float, area: float = 1.0) -> float:
    """R such that a disc of radius R holds about K of M uniformly spread centres."""
    return math.sqrt(K * area / (math.pi * M))


def grid_nodes(n: int, bbox=(0.0, 0.0, 1.0, 1.0)):
    """Node-centred n x n output grid (inclusive linspace on each axis), row-major in y then x.
    Returns (gx, gy) of length n each; node (i, j) is (gx[j], gy[i])."""
    x0, y0, x1, y1 = bbox
    return np.linspace(x0, x1, n), np.linspace(y0, y1, n)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def config_franke(seed: int = 0, N: int = 20_000, M: int = 2_000, K: float = 20.0,
                  kernel: str = "w31", eval_n: int = 256) -> Problem:
    """Uniform points, Franke heights + N(0, 0.01^2) noise, Halton centres (20k x 2k by default)."""
    rng = np.random.default_rng(seed)
    pts = rng.random((N, 2))
    h = franke(pts[:, 0], pts[:, 1]) + rng.normal(0.0, 0.01, N)
    C = halton(M)
    return Problem(pts, h, C, support_radius(M, K), kernel, eval_n=eval_n,
                   name=f"franke_N{N}_M{M}", meta=dict(seed=seed, K=K))


def _gaussian_mixture(rng, N, ncomp=64, sig=(0.01, 0.08), background=0.20):
    means = rng.random((ncomp, 2))
    sigmas = np.exp(rng.uniform(math.log(sig[0]), math.log(sig[1]), ncomp))
    w = rng.random(ncomp)
    w /= w.sum()
    out = np.empty((0, 2))
    while out.shape[0] < N:
        need = N - out.shape[0]
        nb = rng.binomial(need, background)
        bg = rng.random((nb, 2))
        comp = rng.choice(ncomp, size=need - nb, p=w)
        g = means[comp] + sigmas[comp, None] * rng.standard_normal((need - nb, 2))
        cand = np.concatenate([bg, g], axis=0)
        ok = np.all((cand >= 0.0) & (cand < 1.0), axis=1)
        out = np.concatenate([out, cand[ok]], axis=0)
    out = out[:N]
    return out[rng.permutation(N)]


def _bumps(rng, nb=200, s=(0.01, 0.1)):
    m = rng.random((nb, 2))
    a = rng.standard_normal(nb)
    sk = np.exp(rng.uniform(math.log(s[0]), math.log(s[1]), nb))

    def f(x, y):
        out = np.zeros_like(x)
        for k0 in range(0, nb, 25):
            k1 = min(nb, k0 + 25)
            d2 = (x[:, None] - m[None, k0:k1, 0]) ** 2 + (y[:, None] - m[None, k0:k1, 1]) ** 2
            out += (a[None, k0:k1] * np.exp(-d2 / (2.0 * sk[None, k0:k1] ** 2))).sum(axis=1)
        return out
    return f


def config_terrain(seed: int = 0, N: int = 1_000_000, M: int = 100_000, K: float = 30.0,
                   kernel: str = "w31", eval_n: int = 1024) -> Problem:
    """Clustered terrain: 64-Gaussian mixture over a 20 % floor, 200 bumps + value noise
    (1M points x 100k centres by default)."""
    rng = np.random.default_rng(seed)
    pts = _gaussian_mixture(rng, N)
    bumps = _bumps(rng)
    noise = _noise_fn(rng, octaves=6, base=8)
    h = np.empty(N)
    for i0 in range(0, N, 1 << 16):
        i1 = min(N, i0 + (1 << 16))
        x, y = pts[i0:i1, 0], pts[i0:i1, 1]
        h[i0:i1] = bumps(x, y) + 0.1 * noise(x, y)
    C = halton(M)
    return Problem(pts, h, C, support_radius(M, K), kernel, eval_n=eval_n,
                   name=f"terrain_N{N}_M{M}", meta=dict(seed=seed, K=K))


def config_bigdata(seed: int = 0, N: int = 20_000_000, M: int = 2_000_000, K: float = 30.0,
                   kernel: str = "w32", eval_n: int = 4096) -> Problem:
    """Big-data terrain: density 1 + 9 s(x) with s a 3-octave value-noise field scaled to
    [0, 1] (10:1), 8-octave value-noise heights."""
    rng = np.random.default_rng(seed)
    dens = _noise_fn(rng, octaves=3, base=4)
    terr = _noise_fn(rng, octaves=8, base=4)
    # s = the density field scaled to [0, 1] by its range on a 513^2 lattice (finer than its
    # finest octave), so that the density 1 + 9 s varies 10:1
    g = np.linspace(0.0, 1.0, 513)
    GX, GY = np.meshgrid(g, g)
    lat = dens(GX.ravel(), GY.ravel())
    lo, hi = float(lat.min()), float(lat.max())
    chunks, have = [], 0
    while have < N:
        cand = rng.random((1 << 20, 2))
        s = np.clip((dens(cand[:, 0], cand[:, 1]) - lo) / (hi - lo), 0.0, 1.0)
        keep = rng.random(cand.shape[0]) < (1.0 + 9.0 * s) / 10.0
        chunks.append(cand[keep])
        have += int(keep.sum())
    pts = np.concatenate(chunks)[:N]
    h = np.empty(N)
    for i0 in range(0, N, 1 << 20):
        i1 = min(N, i0 + (1 << 20))
        h[i0:i1] = terr(pts[i0:i1, 0], pts[i0:i1, 1])
    C = halton(M)
    return Problem(pts, h, C, support_radius(M, K), kernel, eval_n=eval_n,
                   name=f"bigdata_N{N}_M{M}", meta=dict(seed=seed, K=K))


def tile(seed: int, n_range=(2_000, 200_000), K: float = 30.0, kernel: str = "w31",
         N: int | None = None) -> Problem:
    """One tile of the batched workload (N log-uniform in n_range unless given, M = N // 10)."""
    rng = np.random.default_rng(seed)
    n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
    if N is not None:
        n = int(N)
    m = max(n // 10, 1)
    offset = int(rng.integers(0, 1 << 20))
    pts = rng.random((n, 2))
    s = rng.uniform(0.5, 2.0)
    A = rng.uniform(0.7, 1.3, size=(2, 2)) * np.array([[1.0, 0.3], [0.3, 1.0]]) * rng.choice([-1, 1], 2)
    t = rng.uniform(-0.2, 0.2, size=2)
    u = pts @ A.T + t
    noise = _noise_fn(rng, octaves=4, base=4)
    h = s * franke(u[:, 0], u[:, 1]) + 0.3 * noise(pts[:, 0], pts[:, 1]) + rng.normal(0.0, 0.01, n)
    C = halton(m, start=1 + offset)
    return Problem(pts, h, C, support_radius(m, K), kernel, eval_n=0,
                   name=f"tile_s{seed}_N{n}", meta=dict(seed=seed, K=K))


def tile_batch(first_seed: int, T: int, **kw) -> list:
    """T independent tiles with seeds first_seed .. first_seed+T-1."""
    return [tile(first_seed + t, **kw) for t in range(T)]


def config_small(seed: int, N: int, M: int, K: float = 20.0, kernel: str = "w31",
                 clustered: bool = False, eval_n: int = 33) -> Problem:
    """Small problem for parity tests: uniform (or clustered) points, random centres."""
    rng = np.random.default_rng(seed)
    pts = _gaussian_mixture(rng, N, ncomp=4, sig=(0.05, 0.2), background=0.3) if clustered \
        else rng.random((N, 2))
    h = franke(pts[:, 0], pts[:, 1]) + rng.normal(0.0, 0.01, N)
    C = rng.random((M, 2))
    return Problem(pts, h, C, support_radius(M, K), kernel, eval_n=eval_n,
                   name=f"small_s{seed}_N{N}_M{M}", meta=dict(seed=seed, K=K))


# ----------------------------------------------------------------------------
# warm-start network: seeded initial weights (inputs of both the oracle and the library)
# ----------------------------------------------------------------------------

MLP_NFEAT, MLP_HID = 32, 64
MLP_NPARAM = MLP_HID * MLP_NFEAT + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_HID + 1


def mlp_init(seed: int = 0) -> np.ndarray:
    """Flat FP32 parameters of the 32-64-64-1 network: weights uniform in
    +-sqrt(6 / fan_in) (He), the output layer in +-sqrt(1 / fan_in), biases 0."""
    rng = np.random.default_rng(seed)
    parts = [rng.uniform(-1, 1, (MLP_HID, MLP_NFEAT)) * np.sqrt(6.0 / MLP_NFEAT),
             np.zeros(MLP_HID),
             rng.uniform(-1, 1, (MLP_HID, MLP_HID)) * np.sqrt(6.0 / MLP_HID),
             np.zeros(MLP_HID),
             rng.uniform(-1, 1, MLP_HID) * np.sqrt(1.0 / MLP_HID),
             np.zeros(1)]
    return np.concatenate([a.ravel() for a in parts]).astype(np.float32)
