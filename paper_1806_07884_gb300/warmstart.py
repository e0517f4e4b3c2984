"""Training and use of the warm-start network (host control only: every forward, backward
and Adam step runs in librbf's kernels through ``Context``).

Training data are solved systems: for each centre j its 32 radial features and the target
t_j = c_j / sigma, c the converged least-squares weights and sigma the height scale of the
centre's tile. The network is then used through ``Context.warm_start`` to start
``solve`` / ``solve_tiles`` from c0 = sigma * network(features).
"""
from __future__ import annotations

import os

import numpy as np

from . import Context, pack_tiles

NPARAM = 6337
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "warmstart_w31.npy")


def _torch():
    import torch
    return torch


def training_set(problems, kernel="w31", tol=1e-10, ctx=None, device=0):
    """Features (n, 32) float32 and targets (n,) float32 (CUDA tensors) of the tiles in
    `problems` (sequences (points, h, centres, R, bbox)), fitted together in FP64."""
    torch = _torch()
    dev = f"cuda:{device}"
    tiles, cx, cy, px, py, hh = pack_tiles(problems)
    ctx = ctx or Context(device)
    ctx.bin_tiles(tiles, *[torch.as_tensor(a).to(dev) for a in (cx, cy, px, py, hh)])
    ctx.assemble(kernel, "fp64")
    c, info, tinfo = ctx.solve_tiles(tol=tol)
    feat, _ = ctx.features()
    target = ctx.mlp_targets(c)
    return feat, target, ctx


def train(ctx, feat, target, params=None, epochs=4, batch=4096, lr=2e-3, seed=0,
          lr_final=2e-4, log=None):
    """Adam on mean (y - t)^2 over shuffled minibatches (permutations from a seeded numpy
    generator, passed to the kernels as sample indices). Returns (params, losses)."""
    torch = _torch()
    import datagen as dg   # the seeded initial weights
    dev = feat.device
    n = int(feat.shape[0])
    p = torch.as_tensor(dg.mlp_init(seed) if params is None else params, dtype=torch.float32,
                        device=dev).clone()
    m = torch.zeros(NPARAM, dtype=torch.float32, device=dev)
    v = torch.zeros_like(m)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    rng = np.random.default_rng(seed)
    steps = epochs * max(1, n // batch)
    step = 0
    ctx.mlp_train_step(p, None, None, 0, 0.0, feat, target, n=n, loss=loss)
    losses = [float(loss.item())]          # before training, then after each epoch
    for ep in range(epochs):
        perm = torch.as_tensor(rng.permutation(n).astype(np.int32), device=dev)
        for b0 in range(0, n - batch + 1 if n >= batch else 1, batch):
            idx = perm[b0:b0 + batch]
            step += 1
            frac = min(1.0, step / steps)
            lr_t = lr * (lr_final / lr) ** frac        # geometric decay
            ctx.mlp_train_step(p, m, v, step, lr_t, feat, target, idx=idx, loss=loss)
        # full-set loss of this epoch (gradient-only pass)
        ctx.mlp_train_step(p, None, None, 0, 0.0, feat, target, n=n, loss=loss)
        losses.append(float(loss.item()))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4g}")
    return p, losses


def load_params(path=DEFAULT_WEIGHTS, device=0):
    torch = _torch()
    return torch.as_tensor(np.load(path).astype(np.float32), device=f"cuda:{device}")
