#!/usr/bin/env python3
"""Benchmark of the CS-RBF least-squares fit on GB300: points fitted per second.

One step = the whole hot path on one synthetic workload: bin (a), fused assembly of
B = A^T A and b = A^T h (b, c), Jacobi-PCG solve (d) -- FP32 inner CG with FP64
matrix-free refinement, or plain FP64 -- and evaluation on the output grid (e).
Workload (default): the clustered terrain, N = 1,000,000 points (64-Gaussian mixture
over a 20 % uniform floor), M = 100,000 Halton centres, Wendland phi_{3,1}, about 30
centres per support, 1024 x 1024 output grid, seed = rank.

value      = N / device time per step, inputs resident in HBM, L2 flushed before each
             step (a 512 MiB write).
e2e        = the same through the public API with host inputs: pinned host -> device
             copies of points, heights and centres, the step, device -> host copies of c
             and of the surface f, all inside the timed region.
roofline   = the solver's SpMV kernel (the dominant kernel of the step), algorithmic
             bytes per launch / its mean duration measured with CUDA events on the
             launching stream, against the measured HBM copy bandwidth.
Accuracy   = the surface of the timed path against a tightly converged FP64 solve of the
             same workload (``accuracy`` key), which the GPU parity tests tie to the oracle.

--impl reference runs the CPU FP64 oracle (tests' reference implementation) on a bounded
sample of the same workload instead. Multi-GPU (torchrun): independent replicas (the fit of
one system does not shard), weak scaling.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


# DRAM traffic of the SpMV kernels from ncu captures (the summaries under profiles/), valid
# while the captured kernel's source -- its function text and the shared SpMV device code --
# is unchanged.
CSRC = os.path.join(ROOT, "paper_1806_07884_gb300", "csrc")
# terrain 1M x 100k: read + write of one launch with cold caches (ncu flushes them between
# replays); inside the solve loop the 38 MB of B stay in the 126 MB L2
SPMV_TRAFFIC = {"sha": "a76c524c89379989", "bytes": 37625856 + 0,
                "note": "one launch with cold caches; B is L2-resident inside the solve loop"}
BSPMV_TRAFFIC = {"sha": "0a2682fdead136bb", "per_alg_byte": (230588416 + 5122816) / 148343644}


# The device code every SpMV kernel runs (csrc/rbf_cg.cuh): the row-group record staging, the
# group SpMV and its loads, atomics and butterfly.
SPMV_DEVICE_CODE = ["struct GroupSmem", "void stage_group(", "void group_wait()",
                    "ld4(const float* p)", "ld4(const double* p)", "V4<T>::type ldx4(",
                    "void atomic_add4(", "T butterfly8(", "T spmv_group("]


def _function_text(text, signature):
    """The definition that contains `signature`, from there to its closing brace at column 0
    (or the end of a one-line struct)."""
    i = text.index(signature)
    j = text.index("\n}", i)
    return text[i:j]


def kernel_sha(fname, signature):
    """sha256 (16 hex digits) of the kernel whose definition starts at `signature` in csrc/fname
    together with the SpMV device code it runs from csrc/rbf_cg.cuh."""
    with open(os.path.join(CSRC, fname)) as f:
        text = f.read()
    with open(os.path.join(CSRC, "rbf_cg.cuh")) as f:
        common = f.read()
    parts = [_function_text(text, signature)] + [_function_text(common, sig) for sig in SPMV_DEVICE_CODE]
    return hashlib.sha256("".join(parts).encode()).hexdigest()[:16]


def spmv_traffic():
    ok = SPMV_TRAFFIC["sha"] is not None and \
        kernel_sha("rbf_solve.cu", "k_spmv(Binned bd") == SPMV_TRAFFIC["sha"]
    return SPMV_TRAFFIC["bytes"] if ok else None


# The big-data SpMV is the single-system kernel on a B streamed from HBM; its DRAM traffic per
# algorithmic byte comes from a capture of a smaller big-data system (B still far beyond L2).
BIG_SPMV_TRAFFIC = {"sha": "a76c524c89379989", "per_alg_byte": (189784064 + 4395520) / 121659036,
                    "note": "scaled from a 5M x 500k big-data capture"}


def big_spmv_traffic(alg_bytes):
    ok = BIG_SPMV_TRAFFIC["sha"] is not None and \
        kernel_sha("rbf_solve.cu", "k_spmv(Binned bd") == BIG_SPMV_TRAFFIC["sha"]
    return int(BIG_SPMV_TRAFFIC["per_alg_byte"] * alg_bytes) if ok else None


def bspmv_traffic(alg_bytes):
    ok = kernel_sha("rbf_batch.cu", "k_bcg_spmv(Binned bd") == BSPMV_TRAFFIC["sha"]
    return int(BSPMV_TRAFFIC["per_alg_byte"] * alg_bytes) if ok else None


def spmv_bytes(ctx, M: int, vb: int):
    """Bytes of one SpMV y = B x: the algorithmic bytes of the method (each nonzero of the
    upper triangle of B once, plus three vectors of length M: x read, y read and written) and
    the bytes the library's layout streams (every stored value, 16 B of row description per
    row, 32 B per row group, the same vectors)."""
    st = ctx.layout_stats()
    alg = st["nonzeros"] * vb + 3 * M * vb
    stored = st["stored_values"] * vb + 16 * M + 32 * st["row_groups"] + 3 * M * vb
    return alg, stored, st


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp32_refine", choices=["fp32_refine", "fp64"])
    ap.add_argument("--tol", type=float, default=3e-12)
    ap.add_argument("--N", type=int, default=1_000_000)
    ap.add_argument("--M", type=int, default=100_000)
    ap.add_argument("--grid", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--quiet-extra", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-bigdata", action="store_true")
    ap.add_argument("--bigdata-only", action="store_true",
                    help="run only the big-data workload (its object is the line)")
    ap.add_argument("--big-N", type=int, default=20_000_000)
    ap.add_argument("--big-M", type=int, default=2_000_000)
    ap.add_argument("--big-grid", type=int, default=4096)
    ap.add_argument("--host-b-mb", type=float, default=64.0,
                    help="also time one big-data step with B in host memory, assembled in "
                         "blocks of this many MB (0: skip)")
    ap.add_argument("--inner-tol", type=float, default=1e-2,
                    help="relative tolerance of each FP32 inner solve of the terrain fit (the "
                         "library's default, 1e-3, suits the big-data and batched systems)")
    ap.add_argument("--tiles-inner-tol", type=float, default=None,
                    help="relative tolerance of each FP32 inner solve of the batched tiles "
                         "(default: the library's, 1e-3)")
    ap.add_argument("--windows", type=int, default=4,
                    help="also time the big-data fit as W x W moving windows (0: skip)")
    ap.add_argument("--window-overlap", type=float, default=2.0,
                    help="the windows' overlap in units of R")
    ap.add_argument("--window-margin", type=float, default=2.0,
                    help="the windows' data margin in units of R")
    ap.add_argument("--no-learned", dest="learned", action="store_false",
                    help="cold start instead of the learned warm start in the timed step")
    ap.add_argument("--tiles", type=int, default=512)
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched workload and print its object (profiling)")
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of the ranks' values of x (the slowest rank sets the job's time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Units per second of the whole job: every rank processes units_per_rank in ms."""
    return world * units_per_rank / (ms * 1e-3)


# ----------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax = float(p[1])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if p[4 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------
# the CPU FP64 oracle on a bounded sample (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------------------
def oracle_sample(seed: int, N: int, M: int, tol: float):
    """Time the oracle fit + grid evaluation on a same-statistics sample (N/M = 10, K = 30)."""
    import datagen as dg
    import oracle as O
    pb = dg.config_terrain(seed=seed, N=N, M=M, eval_n=max(32, int(1024 * (N / 1e6) ** 0.5)))
    t0 = time.perf_counter()
    c, _ = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel, tol=tol)
    O.evaluate_grid(c, pb.centres, pb.R, pb.kernel, pb.eval_n)
    return time.perf_counter() - t0, pb


def _oracle_worker(job):
    """One oracle fit in a worker process (single-threaded BLAS): returns its seconds."""
    seed, N, M, tol = job
    return oracle_sample(seed, N, M, tol)[0]


def host_cpu():
    """Logical cores usable by this process and the CPU model name."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return int(cores or 1), model or "unknown"


class OraclePool:
    """Worker processes for the oracle on every host core, started by spawn (never forked
    from a process that has touched CUDA), each with a single BLAS thread."""

    def __init__(self, cores: int):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.cores = cores
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            self.ex = cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"))
            # imports and first-touch of every worker, outside any timing
            list(self.ex.map(_oracle_worker, [(10_000 + k, 5000, 500, 1e-10) for k in range(cores)]))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def rate(self, seeds, N: int, M: int, tol: float):
        """Independent samples fitted concurrently, one per worker: the pool's points per
        second (sum over the workers of N / that worker's fit time) and the mean fit time."""
        ts = list(self.ex.map(_oracle_worker, [(s, N, M, tol) for s in seeds]))
        return sum(N / t for t in ts), statistics.mean(ts)

    def close(self):
        self.ex.shutdown()


def oracle_config1(tol: float):
    """The oracle on the plain FP64 workload at full size (20,000 Franke points, 2,000 Halton
    centres, phi_3,1, 256 x 256 grid), single-threaded: (points/s, seconds)."""
    import datagen as dg
    import oracle as O
    pb = dg.config_franke(seed=0)
    t0 = time.perf_counter()
    c, _ = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel, tol=tol)
    O.evaluate_grid(c, pb.centres, pb.R, pb.kernel, 256)
    t = time.perf_counter() - t0
    return pb.N / t, t


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return
    N, M = 50_000, 5_000
    cores, model = host_cpu()
    pool = OraclePool(cores)
    rates = []
    for k in range(args.warmup + args.steps):
        rate, _ = pool.rate(list(range(100 * k, 100 * k + cores)), N, M, args.tol)
        if k >= args.warmup:
            rates.append(rate)
    pool.close()
    value = statistics.mean(rates)
    sec_per_point = 1.0 / value
    sample = (f"oracle fit (kd-tree, scipy A^T A, Jacobi-PCG tol {args.tol:g}) + grid evaluation of "
              f"the terrain workload at N={N}, M={M} (same N/M and K as 1M x 100k): {cores} "
              f"independent samples per step, one per worker process on {cores} host cores "
              f"({model})")
    line = {"impl": "reference", "metric": "points fitted/s at 1e-6 rel. error, learned+FP32 vs plain FP64", "value": value,
            "unit": "points/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec_per_point * N * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "terrain 1M points x 100k centres, phi_3,1, K=30 (CPU sample)",
                       "N": N, "M": M},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu_model": model},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------
# the GPU path
# ----------------------------------------------------------------------------------------
def bench_batched(args, rank, dev, stream, flush, hbm, peak_source):
    """The batched workload: 512 independent tiles (N log-uniform in [2e3, 2e5], M = N / 10,
    phi_3,1, K = 30) binned, assembled and solved together; sum of N over the fit time."""
    import numpy as np
    import torch

    import datagen as dg
    import paper_1806_07884_gb300 as pkg

    pbs = dg.tile_batch(1000 + 100_000 * rank, args.tiles)
    tiles, cx, cy, px, py, hh = pkg.pack_tiles(
        [(pb.points, pb.h, pb.centres, pb.R, pb.bbox) for pb in pbs])
    d = [torch.as_tensor(a).to(dev) for a in (cx, cy, px, py, hh)]
    Ntot, Mtot = int(px.size), int(cx.size)
    cbuf = torch.empty(Mtot, dtype=torch.float64, device=dev)
    ctx = pkg.Context(dev.index)
    if args.tiles_inner_tol is not None:
        ctx.set_param("inner_tol", args.tiles_inner_tol)

    def step(prec, tol):
        ctx.bin_tiles(tiles, *d)
        ctx.assemble("w31", prec)
        c, info, tinfo = ctx.solve_tiles(tol=tol, maxit=20000, out=cbuf)
        return info, tinfo

    def timed(prec, tol, k):
        ms = []
        gc.collect()
        gc.disable()
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info, tinfo = step(prec, tol)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        gc.enable()
        timed.step_ms = [round(x, 3) for x in ms]
        return statistics.mean(ms), info, tinfo

    for _ in range(2):                     # warm-up (the first one runs the autotuner)
        step(args.prec, args.tol)
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    ms, info, tinfo = timed(args.prec, args.tol, max(2, min(args.steps, 3)))
    launches = (ctx.launch_count() - launches0) // max(2, min(args.steps, 3))
    c_fast = cbuf.clone()
    # roofline of the batched SpMV (every tile running), timed on its stream, on the
    # precision of the timed path (a step that promoted tiles leaves an FP64 B: assemble again)
    if ctx.prec != args.prec:
        step(args.prec, args.tol)
    lay = ctx.layout()
    vb = lay["value_bytes"]
    ctx.bench_spmv(5)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    ctx.bench_spmv(30)
    s1.record(stream)
    torch.cuda.synchronize()
    spmv_ms = s0.elapsed_time(s1) / 30
    alg, stored, lst = spmv_bytes(ctx, Mtot, vb)
    ach = alg / (spmv_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": f"k_bcg_spmv<{'float' if vb == 4 else 'double'}>",
            "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
            "traffic": bspmv_traffic(alg), "traffic_note": "scaled from a 128-tile capture",
            "algorithmic_bytes": alg, "stored_bytes": stored,
            "stored_over_algorithmic": round(stored / alg, 4),
            "upper_nonzeros": lst["nonzeros"], "stored_values": lst["stored_values"],
            "launch_ms": round(spmv_ms, 5), "peak_source": peak_source}
    learned = None
    if args.learned:
        from paper_1806_07884_gb300 import warmstart
        wp = warmstart.load_params(device=dev.index)
        c0b = torch.empty(Mtot, dtype=torch.float64, device=dev)

        def lstep():
            ctx.bin_tiles(tiles, *d)
            ctx.assemble("w31", args.prec)
            c0 = ctx.warm_start(wp, out=c0b)
            return ctx.solve_tiles(tol=args.tol, maxit=20000, c0=c0, out=cbuf)

        lstep()
        lms = []
        for _ in range(2):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, linfo, ltinfo = lstep()
            e1.record(stream)
            e1.synchronize()
            lms.append(e0.elapsed_time(e1))
        learned = {"value": Ntot / (statistics.mean(lms) * 1e-3),
                   "ms_per_step": round(statistics.mean(lms), 3),
                   "iterations_max": linfo["iterations"],
                   "iterations_mean": round(float(np.mean([t["iterations"] for t in ltinfo])), 1),
                   "all_converged": all(t["status"] == 0 for t in ltinfo)}
    tune = ctx.tuning()
    # phases of one step
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    flush.zero_()
    ev[0].record(stream)
    ctx.bin_tiles(tiles, *d)
    ev[1].record(stream)
    ctx.assemble("w31", args.prec)
    ev[2].record(stream)
    ctx.solve_tiles(tol=args.tol, maxit=20000, out=cbuf)
    ev[3].record(stream)
    torch.cuda.synchronize()
    phases = {n: round(ev[k].elapsed_time(ev[k + 1]), 3)
              for k, n in enumerate(["bin", "assemble", "solve"])}
    out = {"workload": f"{args.tiles} tiles, N log-uniform in [2000, 200000], M = N/10, "
                       f"Wendland phi_3,1, K=30, sum N = {Ntot}, sum M = {Mtot}",
           "value": Ntot / (ms * 1e-3), "unit": "points/s", "ms_per_step": round(ms, 3),
           "step_ms": timed.step_ms,
           "prec": args.prec, "tol": args.tol, "inner_tol": args.tiles_inner_tol or 1e-3,
           "gpu_launches_per_step": launches,
           "iterations_max": info["iterations"], "refinements_max": info["refinements"],
           "iterations_mean": round(float(np.mean([t["iterations"] for t in tinfo])), 1),
           "all_converged": all(t["status"] == 0 for t in tinfo), "promoted": info["promoted"],
           "phases_ms": phases, "tuning": tune, "roofline": roof, "learned_start": learned}
    if not args.no_fp64_compare:
        ms64, info64, _ = timed("fp64", args.tol, 1)
        out["fp64_path"] = {"value": Ntot / (ms64 * 1e-3), "ms_per_step": round(ms64, 3),
                            "iterations_max": info64["iterations"]}
        step("fp64", 1e-13)
        c_ref = cbuf.clone()
        # each tile's surface on its own 64 x 64 grid, this path against the tight FP64 fit
        f_fast = ctx.eval_tiles_grid(c_fast, 64, 64).reshape(len(tiles), -1)
        f_ref = ctx.eval_tiles_grid(c_ref, 64, 64).reshape(len(tiles), -1)
        den = f_ref.abs().amax(dim=1).clamp_min(1e-300)
        errs = ((f_fast - f_ref).abs().amax(dim=1) / den).cpu().numpy()
        cerr = []
        for t in tiles:
            a = c_fast[t["c0"]:t["c0"] + t["M"]]
            b = c_ref[t["c0"]:t["c0"] + t["M"]]
            cerr.append(float((a - b).abs().max()) / max(float(b.abs().max()), 1e-300))
        out["accuracy"] = {"max_tile_rel_err_f_vs_fp64_tight": float(errs.max()),
                           "median_tile_rel_err_f": float(np.median(errs)),
                           "max_tile_rel_err_c": max(cerr), "bar": 1e-6,
                           "ok": bool(errs.max() <= 1e-6)}
    ctx.close()
    return out


def bench_host_b(args, ctx, step, timed, N, M, f_dev, fbuf, stream):
    """The same step with B in pinned host memory, assembled in blocks of cell rows that fit
    host_b_mb MB of device memory (Section 5's block-wise assembly, "b_device_mb"); the solver
    reads B over the host link. One step after one warm-up, and the SpMV's rate over the link
    on the stored bytes it reads."""
    import torch

    ctx.set_param("b_device_mb", args.host_b_mb)
    try:
        step(args.prec, args.tol)                   # warm-up
        ms, _, infos = timed(args.prec, args.tol, 1)
        lst = ctx.layout_stats()
        err = float((fbuf - f_dev).abs().max() / f_dev.abs().max())
        vb = ctx.layout()["value_bytes"]
        stored = lst["stored_values"] * vb + 3 * M * vb
        ctx.bench_spmv(2)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        ctx.bench_spmv(10)
        s1.record(stream)
        torch.cuda.synchronize()
        spmv_ms = s0.elapsed_time(s1) / 10
    finally:
        ctx.set_param("b_device_mb", 0.0)
    return {"b_device_mb": args.host_b_mb, "host_blocks": lst["host_blocks"],
            "b_bytes": lst["stored_values"] * vb, "value": N / (ms * 1e-3), "unit": "points/s",
            "ms_per_step": round(ms, 3), "iterations": infos[-1]["iterations"],
            "promoted": int(infos[-1]["promoted"]),
            "spmv_ms": round(spmv_ms, 4),
            "spmv_link_gbs": round(stored / (spmv_ms * 1e-3) / 1e9, 1),
            "rel_err_f_vs_device_b": err, "bar": 1e-6, "ok": err <= 1e-6}


def bench_windows(args, dev, d, pb, f_global, stream, flush):
    """The big-data fit as W x W overlapping windows (the moving window of Section 7): one
    step = bin the windows, assemble and solve them as one batch, evaluate the blended surface
    on the same grid; N over its device time (one warm-up, two timed steps). The blended
    surface is another approximation than the global fit: its difference from it is reported,
    not held to a parity bar (the GPU tests tie both to their oracles)."""
    import torch

    import paper_1806_07884_gb300 as pkg

    W, n = args.windows, args.big_grid
    ov, mg = args.window_overlap * pb.R, args.window_margin * pb.R
    ctx = pkg.Context(dev.index)
    fbuf = torch.empty((n, n), dtype=torch.float64, device=dev)
    box = (0.0, 0.0, 1.0, 1.0)

    def step():
        ctx.bin_windows(*d, pb.R, pb.bbox, W, W, ov, mg)
        ctx.assemble(pb.kernel, args.prec)
        c, info, tinfo = ctx.solve_tiles(tol=args.tol, maxit=50000)
        ctx.eval_windows_grid(c, n, n, box, out=fbuf)
        return c, info, tinfo

    try:
        step()
        torch.cuda.synchronize()
        ms, infos = [], []
        for _ in range(2):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, info, tinfo = step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            infos.append((info, tinfo))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        flush.zero_()
        ev[0].record(stream)
        ctx.bin_windows(*d, pb.R, pb.bbox, W, W, ov, mg)
        ev[1].record(stream)
        ctx.assemble(pb.kernel, args.prec)
        ev[2].record(stream)
        c, _, _ = ctx.solve_tiles(tol=args.tol, maxit=50000)
        ev[3].record(stream)
        ctx.eval_windows_grid(c, n, n, box, out=fbuf)
        ev[4].record(stream)
        torch.cuda.synchronize()
        phases = {nm: round(ev[i].elapsed_time(ev[i + 1]), 3)
                  for i, nm in enumerate(["bin", "assemble", "solve", "eval"])}
        dif = fbuf - f_global
        diff = float(dif.abs().max() / f_global.abs().max())
        rms = float(dif.square().mean().sqrt() / f_global.square().mean().sqrt())
        info, tinfo = infos[-1]
        its = [t["iterations"] for t in tinfo]
        out = {"windows": f"{W}x{W}", "overlap_in_R": args.window_overlap,
               "value": pb.N / (statistics.mean(ms) * 1e-3), "unit": "points/s",
               "ms_per_step": round(statistics.mean(ms), 3), "step_ms": [round(x, 3) for x in ms],
               "margin_in_R": args.window_margin, "phases_ms": phases, "centres_over_M": round(ctx.M / pb.M, 4),
               "points_over_N": round(ctx.N / pb.N, 4),
               "iterations_max": max(its), "iterations_mean": round(sum(its) / len(its), 1),
               "promoted_windows": sum(int(t["promoted"]) for t in tinfo),
               "rel_diff_f_vs_global_fit": diff, "rms_diff_f_vs_global_fit": rms}
    finally:
        ctx.close()
    return out


def bench_bigdata(args, rank, dev, stream, flush, hbm, peak_source):
    """The big-data workload: N = 20 M points with 10:1 density variation, 8-octave value-noise
    heights, M = 2 M Halton centres, Wendland phi_3,2, FP32 assembly and SpMV with FP64
    residual and refinement, 4096 x 4096 evaluation grid; N over the time of one step (bin,
    assemble, solve, evaluate), device-resident inputs, L2 flushed before each step."""
    import numpy as np
    import torch

    import datagen as dg
    import paper_1806_07884_gb300 as pkg

    pb = dg.config_bigdata(seed=rank, N=args.big_N, M=args.big_M, eval_n=args.big_grid)
    N, M, n = pb.N, pb.M, args.big_grid
    d = [torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in
         (pb.centres[:, 0], pb.centres[:, 1], pb.points[:, 0], pb.points[:, 1], pb.h)]
    cbuf = torch.empty(M, dtype=torch.float64, device=dev)
    fbuf = torch.empty((n, n), dtype=torch.float64, device=dev)
    ctx = pkg.Context(dev.index)

    def step(prec, tol):
        ctx.bin(*d, pb.R, pb.bbox)
        ctx.assemble(pb.kernel, prec)
        c, info = ctx.solve(tol=tol, maxit=50000, out=cbuf)
        ctx.eval_grid(c, n, n, out=fbuf)
        return info

    def timed(prec, tol, k):
        ms, infos = [], []
        gc.collect()
        gc.disable()
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(step(prec, tol))
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        gc.enable()
        return statistics.mean(ms), ms, infos

    step(args.prec, args.tol)                       # warm-up
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    k = max(2, min(args.steps, 3))
    ms, step_ms, infos = timed(args.prec, args.tol, k)
    launches = (ctx.launch_count() - launches0) // k
    info = infos[-1]
    f_fast = fbuf.clone()
    # phases of one step
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    flush.zero_()
    ev[0].record(stream)
    ctx.bin(*d, pb.R, pb.bbox)
    ev[1].record(stream)
    ctx.assemble(pb.kernel, args.prec)
    ev[2].record(stream)
    c, _ = ctx.solve(tol=args.tol, maxit=50000, out=cbuf)
    ev[3].record(stream)
    ctx.eval_grid(c, n, n, out=fbuf)
    ev[4].record(stream)
    torch.cuda.synchronize()
    phases = {nm: round(ev[i].elapsed_time(ev[i + 1]), 3)
              for i, nm in enumerate(["bin", "assemble", "solve", "eval"])}
    # roofline of the solver's SpMV (B streamed from HBM at this size), on its stream, on the
    # precision of the timed path (a promoted step leaves an FP64 B: assemble again)
    if ctx.prec != args.prec:
        step(args.prec, args.tol)
    lay = ctx.layout()
    vb = lay["value_bytes"]
    alg, stored, lst = spmv_bytes(ctx, M, vb)
    ctx.bench_spmv(5)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    ctx.bench_spmv(50)
    s1.record(stream)
    torch.cuda.synchronize()
    spmv_ms = s0.elapsed_time(s1) / 50
    ach = alg / (spmv_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": f"k_spmv<{'float' if vb == 4 else 'double'}>",
            "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
            "traffic": big_spmv_traffic(alg), "traffic_note": BIG_SPMV_TRAFFIC["note"],
            "algorithmic_bytes": alg, "stored_bytes": stored,
            "stored_over_algorithmic": round(stored / alg, 4),
            "upper_nonzeros": lst["nonzeros"], "stored_values": lst["stored_values"],
            "launch_ms": round(spmv_ms, 5), "peak_source": peak_source}
    out = {"workload": f"big data: {N} points (10:1 density), {M} Halton centres, Wendland "
                       f"phi_3,2, K=30, {n}x{n} eval grid",
           "value": N / (ms * 1e-3), "unit": "points/s", "ms_per_step": round(ms, 3),
           "step_ms": [round(x, 3) for x in step_ms], "prec": args.prec, "tol": args.tol,
           "gpu_launches_per_step": launches, "iterations": info["iterations"],
           "refinements": info["refinements"],
           "promoted_steps": sum(int(i["promoted"]) for i in infos),
           "phases_ms": phases, "roofline": roof}
    if args.host_b_mb > 0:
        out["out_of_core"] = bench_host_b(args, ctx, step, timed, N, M, f_fast, fbuf, stream)
    if args.windows > 0:
        out["moving_window"] = bench_windows(args, dev, d, pb, f_fast, stream, flush)
    if not args.no_fp64_compare:
        ms64, _, infos64 = timed("fp64", args.tol, 1)
        out["fp64_path"] = {"value": N / (ms64 * 1e-3), "ms_per_step": round(ms64, 3),
                            "iterations": infos64[-1]["iterations"]}
        f_ref = fbuf.clone()
        err = float((f_fast - f_ref).abs().max() / f_ref.abs().max())
        out["accuracy"] = {"rel_err_f_vs_fp64": err, "reference": f"FP64 path at tol {args.tol}",
                           "bar": 1e-6, "ok": err <= 1e-6}
    ctx.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import datagen as dg
    import paper_1806_07884_gb300 as pkg

    rank, local, world = env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    if args.batched_only or args.bigdata_only:
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        run = bench_batched if args.batched_only else bench_bigdata
        out = run(args, rank, dev, torch.cuda.current_stream(dev), flush, hbm,
                  "measured" if "hbm_gbs" in peaks else "fallback")
        if rank == 0:
            print(json.dumps(out), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    pb = dg.config_terrain(seed=rank, N=args.N, M=args.M, eval_n=args.grid)
    N, M, n = pb.N, pb.M, args.grid
    host = {k: torch.as_tensor(np.ascontiguousarray(v)).pin_memory() for k, v in
            dict(cx=pb.centres[:, 0], cy=pb.centres[:, 1], px=pb.points[:, 0],
                 py=pb.points[:, 1], h=pb.h).items()}
    d = {k: v.to(dev) for k, v in host.items()}
    cbuf = torch.empty(M, dtype=torch.float64, device=dev)
    fbuf = torch.empty((n, n), dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ctx = pkg.Context(local)
    if args.inner_tol is not None:
        ctx.set_param("inner_tol", args.inner_tol)
    stream = torch.cuda.current_stream(dev)

    from paper_1806_07884_gb300 import warmstart
    wparams = warmstart.load_params(device=local) if args.learned else None
    c0buf = torch.empty(M, dtype=torch.float64, device=dev)

    def step(inp, prec=args.prec, tol=args.tol, learned=args.learned):
        ctx.bin(inp["cx"], inp["cy"], inp["px"], inp["py"], inp["h"], pb.R, pb.bbox)
        ctx.assemble(pb.kernel, prec)
        c0 = ctx.warm_start(wparams, out=c0buf) if learned else None
        c, info = ctx.solve(tol=tol, maxit=20000, c0=c0, out=cbuf)
        ctx.eval_grid(c, n, n, out=fbuf)
        return info

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- warm-up
    for _ in range(args.warmup):
        flush.zero_()
        info = step(d)
    torch.cuda.synchronize()

    # ---- timed region: K steps, device-resident inputs, L2 flushed before each step
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = ctx.launch_count()
    gc.collect()
    gc.disable()     # no collector pauses inside the host side of the timed steps
    barrier()
    torch.cuda.synchronize()
    step_ms = []
    infos = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos.append(step(d))
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier()
    gc.enable()
    launches = ctx.launch_count() - launches0
    clocks = sampler.stop()
    ms = statistics.mean(step_ms)
    ms = max_over_ranks(ms, world, dev)
    value = whole_job_rate(N, world, ms)

    # ---- per-phase split of one step (not part of the timed number)
    phases = {}
    flush.zero_()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    ev[0].record(stream)
    ctx.bin(d["cx"], d["cy"], d["px"], d["py"], d["h"], pb.R, pb.bbox)
    ev[1].record(stream)
    ctx.assemble(pb.kernel, args.prec)
    ev[2].record(stream)
    c0 = ctx.warm_start(wparams, out=c0buf) if args.learned else None
    ev.append(torch.cuda.Event(enable_timing=True))
    ev[5].record(stream)
    c, info = ctx.solve(tol=args.tol, maxit=20000, c0=c0, out=cbuf)
    ev[3].record(stream)
    ctx.eval_grid(c, n, n, out=fbuf)
    ev[4].record(stream)
    torch.cuda.synchronize()
    phases = {"bin": ev[0].elapsed_time(ev[1]), "assemble": ev[1].elapsed_time(ev[2]),
              "warm_start": ev[2].elapsed_time(ev[5]), "solve": ev[5].elapsed_time(ev[3]),
              "eval": ev[3].elapsed_time(ev[4])}
    phases = {k: round(v, 4) for k, v in phases.items()}

    # ---- roofline of the dominant kernel: the solver's SpMV, timed on its stream
    lay = ctx.layout()
    vb = lay["value_bytes"]
    alg, stored, lst = spmv_bytes(ctx, M, vb)
    reps = 200
    ctx.bench_spmv(10)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    ctx.bench_spmv(reps)
    s1.record(stream)
    torch.cuda.synchronize()
    spmv_ms = s0.elapsed_time(s1) / reps
    # one CG iteration (SpMV + update kernels) launched individually, same workspace
    ctx.bench_cg(10)
    s0.record(stream)
    ctx.bench_cg(100)
    s1.record(stream)
    torch.cuda.synchronize()
    cg_iter_us = s0.elapsed_time(s1) * 1e3 / 100
    # the solver's own loop (one cooperative launch of the persistent kernel here)
    ctx.bench_cg_loop(50)
    s0.record(stream)
    ctx.bench_cg_loop(500)
    s1.record(stream)
    torch.cuda.synchronize()
    cg_loop_us = s0.elapsed_time(s1) * 1e3 / 500
    achieved = alg / (spmv_ms * 1e-3) / 1e9
    # L2 ceiling: the terrain's stored B fits in the 126 MB L2, so its SpMV streams from L2;
    # a plain device copy of a 24 MiB buffer (read + write 48 MiB, resident in L2), timed
    # like the SpMV, gives the rate L2 sustains for a stream
    l2a = torch.empty(24 << 20, dtype=torch.uint8, device=dev)
    l2b = torch.empty_like(l2a)
    for _ in range(20):
        l2b.copy_(l2a)
    s0.record(stream)
    for _ in range(200):
        l2b.copy_(l2a)
    s1.record(stream)
    torch.cuda.synchronize()
    l2_gbs = 2 * l2a.numel() / (s0.elapsed_time(s1) * 1e-3 / 200) / 1e9
    del l2a, l2b
    roofline = {"bound": "hbm", "kernel": f"k_spmv<{'float' if vb == 4 else 'double'}>",
                "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": spmv_traffic(),
                "traffic_note": SPMV_TRAFFIC["note"],
                "algorithmic_bytes": alg, "stored_bytes": stored,
                "stored_over_algorithmic": round(stored / alg, 4),
                "upper_nonzeros": lst["nonzeros"], "stored_values": lst["stored_values"],
                "launch_ms": round(spmv_ms, 5),
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "cg_iteration_us_plain_launches": round(cg_iter_us, 2),
                "cg_iteration_us_solver_loop": round(cg_loop_us, 2),
                "l2": {"peak": round(l2_gbs, 1), "unit": "GB/s",
                       "frac": round(achieved / l2_gbs, 4),
                       "peak_source": "measured in this run: device copy of 24 MiB, read + write",
                       "b_fits_in_l2": stored < 100e6}}

    # ---- FMA peaks of this GPU, measured in this run, and the FP64 refinement residual
    def fma_tflops(prec, reps):
        ctx.bench_fma(prec, max(1, reps // 8))
        s0.record(stream)
        fl = ctx.bench_fma(prec, reps)
        s1.record(stream)
        torch.cuda.synchronize()
        return fl / (s0.elapsed_time(s1) * 1e-3) / 1e12
    fma = {"fp32_tflops": round(fma_tflops("fp32_refine", 1 << 16), 2),
           "fp64_tflops": round(fma_tflops("fp64", 1 << 12), 3),
           "source": "measured in this run: 8 independent FMA chains per thread, 8 blocks of "
                     "256 threads per SM (rbf_bench_fma)"}
    alu = []
    if args.prec == "fp32_refine":
        # A's nonzeros = the support counts summed (pairs with ||x_i - xi_j|| < R)
        sup = ctx.export_upper()[4]
        nnz_a = int(sup.sum().item())
        del sup
        ctx.bench_residual(2)
        s0.record(stream)
        ctx.bench_residual(10)
        s1.record(stream)
        torch.cuda.synchronize()
        res_ms = s0.elapsed_time(s1) / 10
        fl = 4.0 * nnz_a          # A c and A^T e: one FMA per nonzero each
        ach = fl / (res_ms * 1e-3) / 1e12
        alu.append({"kernel": "k_residual_stored (FP64 refinement residual r = A^T (h - A x))",
                    "bound": "fp64", "achieved": round(ach, 3), "peak": fma["fp64_tflops"],
                    "unit": "TFLOP/s", "frac": round(ach / fma["fp64_tflops"], 4),
                    "flops_per_launch": fl, "model": "4 flops per nonzero of A (A c, A^T e)",
                    "a_nonzeros": nnz_a, "launch_ms": round(res_ms, 4),
                    "stored_a_bytes_per_launch": 8 * nnz_a})
    # the evaluation grid: pairs (node, centre within R) ~ nodes x M pi R^2 / area
    area = (pb.bbox[2] - pb.bbox[0]) * (pb.bbox[3] - pb.bbox[1])
    pairs = n * n * M * np.pi * pb.R ** 2 / area
    fl = 19.0 * pairs
    ach = fl / (phases["eval"] * 1e-3) / 1e12
    alu.append({"kernel": f"k_eval_grid ({n}^2 nodes, FP64 Wendland sums)", "bound": "fp64",
                "achieved": round(ach, 3), "peak": fma["fp64_tflops"], "unit": "TFLOP/s",
                "frac": round(ach / fma["fp64_tflops"], 4), "flops_per_launch": round(fl),
                "model": "19 FP64 flops per node-centre pair in support (difference, r^2, "
                         "square root, Wendland polynomial, accumulation); pairs estimated as "
                         "nodes x M pi R^2 / area", "pairs": round(pairs),
                "launch_ms": phases["eval"]})

    # ---- accuracy: this path's surface against a tight FP64 solve of the same workload
    f_fast = fbuf.clone()
    acc = {}
    fp64 = None
    other = None
    if not args.no_fp64_compare:
        # the same precision with the other start (cold if the timed step is learned)
        o_ms = []
        for _ in range(max(2, min(args.steps, 3))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            info_o = step(d, learned=not args.learned)
            t1.record(stream)
            torch.cuda.synchronize()
            o_ms.append(t0.elapsed_time(t1))
        oms = statistics.mean(o_ms)
        other = {"start": "cold" if args.learned else "learned", "value": N / (oms * 1e-3),
                 "ms_per_step": round(oms, 3), "iterations": info_o["iterations"],
                 "refinements": info_o["refinements"]}
    if not args.no_fp64_compare:
        flush.zero_()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        info64 = step(d, prec="fp64", tol=args.tol)
        t1.record(stream)
        torch.cuda.synchronize()
        fp64_ms = t0.elapsed_time(t1)
        fp64 = {"value": N / (fp64_ms * 1e-3), "ms_per_step": round(fp64_ms, 3),
                "iterations": info64["iterations"], "tol": args.tol}
        # the FP64 path's SpMV, on the FP64 B this step assembled: 2 FMA per off-diagonal
        # stored nonzero (row and column products), 1 per diagonal one
        if ctx.prec == "fp64":
            ctx.bench_spmv(5)
            s0.record(stream)
            ctx.bench_spmv(50)
            s1.record(stream)
            torch.cuda.synchronize()
            sp64_ms = s0.elapsed_time(s1) / 50
            fl = 4.0 * (lst["nonzeros"] - M) + 2.0 * M
            ach = fl / (sp64_ms * 1e-3) / 1e12
            alu.append({"kernel": "k_spmv<double> (FP64 path)", "bound": "fp64",
                        "achieved": round(ach, 3), "peak": fma["fp64_tflops"], "unit": "TFLOP/s",
                        "frac": round(ach / fma["fp64_tflops"], 4), "flops_per_launch": fl,
                        "model": "4 flops per off-diagonal upper nonzero, 2 per diagonal",
                        "launch_ms": round(sp64_ms, 4),
                        "bytes_per_launch": 8 * lst["stored_values"] + 3 * 8 * M})
        step(d, prec="fp64", tol=1e-13)
        f_ref = fbuf.clone()
        err = float((f_fast - f_ref).abs().max() / f_ref.abs().max())
        acc = {"rel_err_f_vs_fp64_tight": err, "bar": 1e-6, "ok": err <= 1e-6}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        c_host = torch.empty(M, dtype=torch.float64).pin_memory()
        f_host = torch.empty((n, n), dtype=torch.float64).pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = c_host.numel() * 8 + f_host.numel() * 8
        e_ms = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dd = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
            step(dd)
            c_host.copy_(cbuf, non_blocking=True)
            f_host.copy_(fbuf, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            e_ms.append(e0.elapsed_time(e1))
        ems = statistics.mean(e_ms)
        ems = max_over_ranks(ems, world, dev)
        e2e = {"value": whole_job_rate(N, world, ems), "unit": "points/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": round(ems, 3)}

    # ---- the batched workload (its own sub-object of the line)
    batched = None
    if not args.no_batched:
        batched = bench_batched(args, rank, dev, stream, flush, hbm,
                                "measured" if "hbm_gbs" in peaks else "fallback")

    # ---- the big-data workload (its own sub-object of the line)
    bigdata = None
    if not args.no_bigdata:
        bigdata = bench_bigdata(args, rank, dev, stream, flush, hbm,
                                "measured" if "hbm_gbs" in peaks else "fallback")

    # ---- CPU baseline: the oracle on bounded samples (rank 0, single GPU only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores, model = host_cpu()
        Ns, Ms = 100_000, 10_000
        t, pbs = oracle_sample(seed=0, N=Ns, M=Ms, tol=args.tol)
        pool = OraclePool(cores)
        rate_all, tmean = pool.rate(list(range(1, cores + 1)), Ns, Ms, args.tol)
        pool.close()
        r1, t1 = oracle_config1(args.tol)
        cpu = {"value": rate_all, "unit": "points/s", "cores": cores, "kind": "oracle",
               "sample": f"{cores} independent samples of the terrain workload at N={Ns}, M={Ms} "
                         f"(same N/M, K; fit + {pbs.eval_n}^2 grid eval), one per worker process "
                         f"on all {cores} host cores ({tmean:.1f} s per fit)",
               "cpu_model": model, "nproc": cores,
               "single_core": {"value": Ns / t, "unit": "points/s", "cores": 1,
                               "sample": f"one such sample, {t:.1f} s single-threaded"},
               "plain_fp64_config_full": {"value": r1, "unit": "points/s", "cores": 1,
                                          "sample": "20,000 Franke points x 2,000 Halton centres, "
                                                    f"phi_3,1, 256^2 grid, full size, {t1:.2f} s "
                                                    "single-threaded"}}

    if rank == 0:
        last = infos[-1]
        line = {
            "metric": "points fitted/s at 1e-6 rel. error, learned+FP32 vs plain FP64",
            "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("bf16/f32 net + " if args.learned else "") +
                     ("f32+f64" if args.prec == "fp32_refine" else "f64"),
            "data": "synthetic",
            "config": {"workload": f"terrain {N} points x {M} Halton centres, Wendland phi_3,1, "
                                   f"K=30, {n}x{n} eval grid",
                       "N": N, "M": M, "kernel": pb.kernel, "prec": args.prec, "tol": args.tol,
                       "inner_tol": args.inner_tol if args.inner_tol is not None else 1e-3,
                       "warm_start": "learned (32-64-64-1 network, paper_1806_07884_gb300/"
                                     "warmstart_w31.npy)" if args.learned else "none",
                       "l2": "flushed before each step (512 MiB write)",
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
            "fma_peaks": fma, "alu_rooflines": alu,
            "clocks": clocks, "accuracy": acc, "fp64_path": fp64, "other_start": other,
            "phases_ms": phases,
            "batched": batched,
            "bigdata": bigdata,
            "solver": {"iterations": last["iterations"], "refinements": last["refinements"],
                       "rel_residual": last["rel_residual"], "pinned": last["pinned"],
                       "promoted_steps": sum(int(i["promoted"]) for i in infos)},
            "step_ms": [round(x, 3) for x in step_ms],
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
