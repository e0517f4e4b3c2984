"""Train the warm-start network on systems the method itself solves, and report its gain.

    python -m paper_1806_07884_gb300.train_warmstart --out paper_1806_07884_gb300/warmstart_w31.npy

Training systems: tiles of the batched workload (seeds 100000 + k, N log-uniform in
[2e3, 2e5], M = N / 10, phi_3,1) and full-size clustered terrains (seeds 1, 2, ...; the
benchmark's terrain is seed 0), each solved in FP64 to a 1e-10 normal residual. Samples are
the centres: 32 radial features, target c_j / sigma. Held out: tiles with seeds 900000 + k
and the terrain of seed 0, solved cold and warm-started (FP32 + FP64 refinement); the
report gives CG iterations and solve times of both. Every step runs in librbf's kernels.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--tiles", type=int, default=10000)
    ap.add_argument("--terrain", type=int, default=4, help="full-size terrains for training")
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--eval-tiles", type=int, default=512)
    ap.add_argument("--tol", type=float, default=3e-12)
    ap.add_argument("--out", required=True)
    args = ap.parse_args()

    import torch

    import datagen as dg
    import paper_1806_07884_gb300 as pkg
    from paper_1806_07884_gb300 import warmstart as W

    dev = "cuda:0"
    t0 = time.time()
    ctx = pkg.Context()
    feats, targets = [], []
    for k0 in range(0, args.tiles, 512):
        pbs = dg.tile_batch(100_000 + k0, min(512, args.tiles - k0))
        f, t, _ = W.training_set([(p.points, p.h, p.centres, p.R, p.bbox) for p in pbs], ctx=ctx)
        feats.append(f)
        targets.append(t)
    for s in range(1, args.terrain + 1):
        pb = dg.config_terrain(seed=s)
        d = [torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in
             (pb.centres[:, 0], pb.centres[:, 1], pb.points[:, 0], pb.points[:, 1], pb.h)]
        ctx.bin(*d, pb.R, pb.bbox)
        ctx.assemble(pb.kernel, "fp64")
        c, info = ctx.solve(tol=1e-10, maxit=50000)
        f, sig = ctx.features()
        feats.append(f)
        targets.append((c / sig[0]).float())
    F = torch.cat(feats)
    T = torch.cat(targets)
    t_data = time.time() - t0
    t1 = time.time()
    params, losses = W.train(ctx, F, T, epochs=args.epochs, batch=args.batch, lr=args.lr,
                             seed=args.seed)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    np.save(args.out, params.cpu().numpy())
    ctx.close()

    # held-out tiles: cold vs warm start, FP32 + FP64 refinement
    pbs = dg.tile_batch(900_000, args.eval_tiles)
    tiles, cx, cy, px, py, hh = pkg.pack_tiles([(p.points, p.h, p.centres, p.R, p.bbox) for p in pbs])
    d = [torch.as_tensor(a).to(dev) for a in (cx, cy, px, py, hh)]
    ctx = pkg.Context()
    ctx.bin_tiles(tiles, *d)
    ctx.assemble("w31", "fp32_refine")
    res = {}
    for name in ("cold", "warm", "cold", "warm"):         # second round timed warm
        torch.cuda.synchronize()
        e0 = time.time()
        c0 = ctx.warm_start(params) if name == "warm" else None
        c, info, tinfo = ctx.solve_tiles(tol=args.tol, c0=c0)
        torch.cuda.synchronize()
        res[name] = {"ms": round(1e3 * (time.time() - e0), 2),
                     "iterations_sum": sum(t["iterations"] for t in tinfo),
                     "iterations_max": info["iterations"], "refinements_max": info["refinements"]}
    ctx.close()
    # the terrain of seed 0 (the benchmark's workload)
    pb = dg.config_terrain(seed=0)
    d = [torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in
         (pb.centres[:, 0], pb.centres[:, 1], pb.points[:, 0], pb.points[:, 1], pb.h)]
    ctx = pkg.Context()
    ctx.bin(*d, pb.R, pb.bbox)
    ctx.assemble(pb.kernel, "fp32_refine")
    ter = {}
    for name in ("cold", "warm", "cold", "warm"):
        torch.cuda.synchronize()
        e0 = time.time()
        c0 = ctx.warm_start(params) if name == "warm" else None
        c, info = ctx.solve(tol=args.tol, c0=c0, maxit=20000)
        torch.cuda.synchronize()
        ter[name] = {"ms": round(1e3 * (time.time() - e0), 2), "iterations": info["iterations"],
                     "refinements": info["refinements"]}
    ctx.close()
    print(json.dumps({"samples": int(F.shape[0]), "data_s": round(t_data, 1),
                      "train_s": round(t_train, 1), "losses": [round(x, 5) for x in losses],
                      "target_var": float(T.double().var()), "held_out_tiles": res,
                      "terrain_seed0": ter}), flush=True)


if __name__ == "__main__":
    main()
