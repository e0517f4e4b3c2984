"""GB300-native compactly supported RBF least-squares surface approximation.

A thin Python layer over the C-ABI library librbf (include/rbf.h). PyTorch supplies
device memory (through the caching allocator, wired in as librbf's workspace
allocator) and streams; every step of the method runs in the library's CUDA kernels:

    ctx = Context()
    ctx.bin(centres, points, h, R, bbox)      # step (a): uniform cell grid of side R
    ctx.assemble("w31", "fp64")               # steps (b)+(c): B = A^T A, b = A^T h (Eq. 11-12)
    c, info = ctx.solve(tol=1e-10)            # step (d): Jacobi-PCG (+ FP64 refinement)
    f = ctx.eval_grid(c, 256, 256)            # step (e): f = sum_j c_j phi(|x - xi_j| / R) (Eq. 3)

``fit`` runs the whole path in one call. Coordinates, heights and weights are float64.
"""
from __future__ import annotations

import ctypes as C

from . import _lib
from ._lib import KERNELS, PRECS, RBFError

__all__ = ["Context", "fit", "fit_poly", "fit_tiles", "pack_tiles", "RBFError", "KERNELS",
           "PRECS", "max_candidates"]


def _torch():
    import torch
    return torch


def max_candidates() -> int:
    return int(_lib.load().rbf_max_candidates())


def _dptr(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


class Context:
    """One librbf context on one CUDA device (not thread-safe)."""

    def __init__(self, device: int = 0, torch_allocator: bool = True):
        torch = _torch()
        self.lib = _lib.load()
        self.device = int(device)
        if torch_allocator:
            dev = self.device

            def _alloc(nbytes, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
                except Exception:       # out of memory: the library reports RBF_ERR_ALLOC
                    return None

            def _free(ptr, nbytes, stream, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._alloc = _lib.ALLOC_FN(_alloc)
            self._free = _lib.FREE_FN(_free)
        else:
            self._alloc = C.cast(None, _lib.ALLOC_FN)
            self._free = C.cast(None, _lib.FREE_FN)
        h = C.c_void_p()
        s = self.lib.rbf_create(C.byref(h), self.device, self._alloc, self._free, None)
        if s != 0:
            raise RBFError(s, "rbf_create failed")
        self._h = h
        self.M = self.N = self.T = 0
        self.kernel = None
        self.prec = None

    # -- plumbing ---------------------------------------------------------------------
    def _check(self, status: int, what: str):
        if status != 0:
            msg = self.lib.rbf_last_error(self._h)
            raise RBFError(status, f"{what}: {msg.decode() if msg else ''}")

    def _stream(self, stream):
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.rbf_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- steps --------------------------------------------------------------------------
    def bin(self, cx, cy, px, py, h, R: float, bbox=(0.0, 0.0, 1.0, 1.0), stream=None):
        """Step (a). cx, cy: M centre coordinates; px, py, h: N points and heights (CUDA float64)."""
        M, N = int(cx.numel()), int(px.numel())
        box = (C.c_double * 4)(*[float(v) for v in bbox])
        s = self.lib.rbf_bin(self._h, _dptr(cx, "cx"), _dptr(cy, "cy"), M, _dptr(px, "px"),
                             _dptr(py, "py"), _dptr(h, "h"), N, float(R), box,
                             self._stream(stream))
        self._check(s, "rbf_bin")
        self.M, self.N, self.T = M, N, 0

    def assemble(self, kernel: str = "w31", prec: str = "fp64", stream=None):
        """Steps (b)+(c): fused rows of A and B = A^T A, b = A^T h."""
        s = self.lib.rbf_assemble(self._h, KERNELS[kernel], PRECS[prec], self._stream(stream))
        self._check(s, "rbf_assemble")
        self.kernel, self.prec = kernel, prec

    def solve(self, tol: float = 1e-10, maxit: int = 100000, min_support: int = 3, c0=None,
              out=None, stream=None, raise_on_fail: bool = True):
        """Step (d): returns (c, info). c0: optional warm start (CUDA float64, length M)."""
        torch = _torch()
        c = out if out is not None else torch.empty(self.M, dtype=torch.float64,
                                                    device=f"cuda:{self.device}")
        if c0 is not None and c0.data_ptr() != c.data_ptr():
            c.copy_(c0)
        info = _lib.SolveInfo()
        s = self.lib.rbf_solve(self._h, _dptr(c, "c"), 1 if c0 is not None else 0, float(tol),
                               int(maxit), int(min_support), C.byref(info), self._stream(stream))
        d = dict(iterations=info.iterations, refinements=info.refinements,
                 rel_residual=info.rel_residual, pinned=info.pinned, promoted=info.promoted,
                 status=s)
        if info.promoted:
            self.prec = "fp64"
        if s != 0 and raise_on_fail:
            self._check(s, "rbf_solve")
        return c, d

    def eval(self, c, qx, qy, out=None, stream=None):
        """Step (e) at query points."""
        torch = _torch()
        Q = int(qx.numel())
        f = out if out is not None else torch.empty(Q, dtype=torch.float64, device=qx.device)
        s = self.lib.rbf_eval(self._h, _dptr(c, "c"), _dptr(qx, "qx"), _dptr(qy, "qy"), Q,
                              _dptr(f, "f"), self._stream(stream))
        self._check(s, "rbf_eval")
        return f

    def eval_grid(self, c, nx: int, ny: int, box=(0.0, 0.0, 1.0, 1.0), out=None, stream=None):
        """Step (e) on the node-centred nx x ny grid; returns f with shape (ny, nx)."""
        torch = _torch()
        f = out if out is not None else torch.empty((ny, nx), dtype=torch.float64, device=c.device)
        b = (C.c_double * 4)(*[float(v) for v in box])
        s = self.lib.rbf_eval_grid(self._h, _dptr(c, "c"), int(nx), int(ny), b, _dptr(f, "f"),
                                   self._stream(stream))
        self._check(s, "rbf_eval_grid")
        return f

    # -- linear polynomial reproduction (Section 3, Eq. 6-10) ------------------------------
    def assemble_poly(self, kernel: str = "w31", prec: str = "fp64", stream=None):
        """Steps (b)+(c) with the polynomial blocks of Eq. 10 (A^T P, P^T P, P^T h)."""
        s = self.lib.rbf_assemble_poly(self._h, KERNELS[kernel], PRECS[prec], self._stream(stream))
        self._check(s, "rbf_assemble_poly")
        self.kernel, self.prec = kernel, prec

    def solve_poly(self, tol: float = 1e-10, maxit: int = 100000, min_support: int = 3,
                   out=None, kout=None, stream=None, raise_on_fail: bool = True):
        """Step (d) on the bordered system of Eq. 10: returns (c, k, info), k = (a_x, a_y, a_0)
        in the caller's coordinates (CUDA float64, length 3)."""
        torch = _torch()
        dev = f"cuda:{self.device}"
        c = out if out is not None else torch.empty(self.M, dtype=torch.float64, device=dev)
        k = kout if kout is not None else torch.empty(3, dtype=torch.float64, device=dev)
        info = _lib.SolveInfo()
        s = self.lib.rbf_solve_poly(self._h, _dptr(c, "c"), _dptr(k, "k"), float(tol), int(maxit),
                                    int(min_support), C.byref(info), self._stream(stream))
        d = dict(iterations=info.iterations, refinements=info.refinements,
                 rel_residual=info.rel_residual, pinned=info.pinned, promoted=info.promoted,
                 status=s)
        if info.promoted:
            self.prec = "fp64"
        if s != 0 and raise_on_fail:
            self._check(s, "rbf_solve_poly")
        return c, k, d

    def eval_poly(self, c, k, qx, qy, out=None, stream=None):
        """Step (e) with the polynomial at query points."""
        torch = _torch()
        Q = int(qx.numel())
        f = out if out is not None else torch.empty(Q, dtype=torch.float64, device=qx.device)
        s = self.lib.rbf_eval_poly(self._h, _dptr(c, "c"), _dptr(k, "k"), _dptr(qx, "qx"),
                                   _dptr(qy, "qy"), Q, _dptr(f, "f"), self._stream(stream))
        self._check(s, "rbf_eval_poly")
        return f

    def eval_grid_poly(self, c, k, nx: int, ny: int, box=(0.0, 0.0, 1.0, 1.0), out=None,
                       stream=None):
        """Step (e) with the polynomial on the node-centred nx x ny grid; shape (ny, nx)."""
        torch = _torch()
        f = out if out is not None else torch.empty((ny, nx), dtype=torch.float64, device=c.device)
        b = (C.c_double * 4)(*[float(v) for v in box])
        s = self.lib.rbf_eval_grid_poly(self._h, _dptr(c, "c"), _dptr(k, "k"), int(nx), int(ny),
                                        b, _dptr(f, "f"), self._stream(stream))
        self._check(s, "rbf_eval_grid_poly")
        return f

    # -- batched tiles --------------------------------------------------------------------
    def bin_tiles(self, tiles, cx, cy, px, py, h, stream=None):
        """Batched step (a). tiles: sequence of dicts {c0, M, p0, N, R, bbox}; cx, cy, px, py,
        h: concatenated CUDA float64 arrays (see rbf_bin_tiles)."""
        T = len(tiles)
        arr = (_lib.Tile * T)()
        for k, t in enumerate(tiles):
            arr[k].c0, arr[k].M = int(t["c0"]), int(t["M"])
            arr[k].p0, arr[k].N = int(t["p0"]), int(t["N"])
            arr[k].R = float(t["R"])
            for q in range(4):
                arr[k].bbox[q] = float(t["bbox"][q])
        M, N = int(cx.numel()), int(px.numel())
        nul = C.c_void_p()
        s = self.lib.rbf_bin_tiles(self._h, arr, T, _dptr(cx, "cx"), _dptr(cy, "cy"), M,
                                   _dptr(px, "px") if N else nul, _dptr(py, "py") if N else nul,
                                   _dptr(h, "h") if N else nul, N, self._stream(stream))
        self._check(s, "rbf_bin_tiles")
        self.M, self.N, self.T = M, N, T

    def solve_tiles(self, tol: float = 1e-10, maxit: int = 100000, min_support: int = 3,
                    c0=None, out=None, stream=None, raise_on_fail: bool = True):
        """Batched step (d): returns (c, info, per-tile info list)."""
        torch = _torch()
        c = out if out is not None else torch.empty(self.M, dtype=torch.float64,
                                                    device=f"cuda:{self.device}")
        if c0 is not None and c0.data_ptr() != c.data_ptr():
            c.copy_(c0)
        T = self.T
        tinfo = (_lib.TileInfo * T)()
        info = _lib.SolveInfo()
        s = self.lib.rbf_solve_tiles(self._h, _dptr(c, "c"), 1 if c0 is not None else 0,
                                     float(tol), int(maxit), int(min_support), tinfo,
                                     C.byref(info), self._stream(stream))
        d = dict(iterations=info.iterations, refinements=info.refinements,
                 rel_residual=info.rel_residual, pinned=info.pinned, promoted=info.promoted,
                 status=s)
        tl = [dict(iterations=t.iterations, refinements=t.refinements,
                   rel_residual=t.rel_residual, pinned=t.pinned, status=t.status,
                   promoted=t.promoted) for t in tinfo]
        if info.promoted:
            self.prec = "fp64"
        if s != 0 and raise_on_fail:
            self._check(s, "rbf_solve_tiles")
        return c, d, tl

    def eval_tiles(self, c, qx, qy, qoff, out=None, stream=None):
        """Batched step (e) at queries grouped by tile: tile t's queries are
        qx[qoff[t]:qoff[t+1]] (qoff: T+1 host integers)."""
        torch = _torch()
        Q = int(qx.numel())
        f = out if out is not None else torch.empty(Q, dtype=torch.float64, device=qx.device)
        off = (C.c_int64 * (self.T + 1))(*[int(v) for v in qoff])
        s = self.lib.rbf_eval_tiles(self._h, _dptr(c, "c"), _dptr(qx, "qx"), _dptr(qy, "qy"),
                                    off, _dptr(f, "f"), self._stream(stream))
        self._check(s, "rbf_eval_tiles")
        return f

    def eval_tiles_grid(self, c, nx: int, ny: int, out=None, stream=None):
        """Batched step (e) on each tile's nx x ny node grid over its bbox: shape (T, ny, nx)."""
        torch = _torch()
        f = out if out is not None else torch.empty((self.T, ny, nx), dtype=torch.float64,
                                                    device=c.device)
        s = self.lib.rbf_eval_tiles_grid(self._h, _dptr(c, "c"), int(nx), int(ny), _dptr(f, "f"),
                                         self._stream(stream))
        self._check(s, "rbf_eval_tiles_grid")
        return f

    # -- moving window ----------------------------------------------------------------------
    def bin_windows(self, cx, cy, px, py, h, R: float, bbox, wx: int, wy: int, overlap: float,
                    margin: float | None = None, stream=None):
        """Lay out wx x wy overlapping windows over bbox and bin them as a batch (see
        rbf_bin_windows; margin defaults to R); then assemble and solve_tiles fit every
        window."""
        M, N = int(cx.numel()), int(px.numel())
        box = (C.c_double * 4)(*[float(v) for v in bbox])
        m = float(R if margin is None else margin)
        s = self.lib.rbf_bin_windows(self._h, _dptr(cx, "cx"), _dptr(cy, "cy"), M, _dptr(px, "px"),
                                     _dptr(py, "py"), _dptr(h, "h"), N, float(R), box, int(wx),
                                     int(wy), float(overlap), m, self._stream(stream))
        self._check(s, "rbf_bin_windows")
        mt, nt = C.c_int64(), C.c_int64()
        self._check(self.lib.rbf_window_sizes(self._h, C.byref(mt), C.byref(nt)), "rbf_window_sizes")
        self.M, self.N, self.T = mt.value, nt.value, int(wx) * int(wy)

    def window_centres(self, stream=None):
        """Input index of the centre behind each of the windows' Mtot weights (CUDA int64)."""
        torch = _torch()
        idx = torch.empty(self.M, dtype=torch.int64, device=f"cuda:{self.device}")
        self._check(self.lib.rbf_window_centres(self._h, C.c_void_p(idx.data_ptr()), self.M,
                                                self._stream(stream)), "rbf_window_centres")
        return idx

    def eval_windows(self, c, qx, qy, out=None, stream=None):
        """The blended moving-window surface at query points."""
        torch = _torch()
        Q = int(qx.numel())
        f = out if out is not None else torch.empty(Q, dtype=torch.float64, device=qx.device)
        self._check(self.lib.rbf_eval_windows(self._h, _dptr(c, "c"), _dptr(qx, "qx"),
                                              _dptr(qy, "qy"), Q, _dptr(f, "f"),
                                              self._stream(stream)), "rbf_eval_windows")
        return f

    def eval_windows_grid(self, c, nx: int, ny: int, box=(0.0, 0.0, 1.0, 1.0), out=None,
                          stream=None):
        """The blended moving-window surface on the nx x ny node grid over box, shape (ny, nx)."""
        torch = _torch()
        f = out if out is not None else torch.empty((ny, nx), dtype=torch.float64, device=c.device)
        b = (C.c_double * 4)(*[float(v) for v in box])
        self._check(self.lib.rbf_eval_windows_grid(self._h, _dptr(c, "c"), int(nx), int(ny), b,
                                                   _dptr(f, "f"), self._stream(stream)),
                    "rbf_eval_windows_grid")
        return f

    # -- learned warm start ----------------------------------------------------------------
    def features(self, out=None, stream=None):
        """Radial features of every centre (caller order, (M, 32) float32 CUDA tensor) and the
        height scale(s) sigma (T or 1 values)."""
        torch = _torch()
        dev = f"cuda:{self.device}"
        f = out if out is not None else torch.empty((self.M, 32), dtype=torch.float32, device=dev)
        sig = torch.empty(max(self.T, 1), dtype=torch.float64, device=dev)
        s = self.lib.rbf_features(self._h, C.c_void_p(f.data_ptr()), C.c_void_p(sig.data_ptr()),
                                  self._stream(stream))
        self._check(s, "rbf_features")
        return f, sig

    def mlp_forward(self, params, feat, out=None, stream=None):
        torch = _torch()
        n = int(feat.shape[0])
        y = out if out is not None else torch.empty(n, dtype=torch.float32, device=feat.device)
        s = self.lib.rbf_mlp_forward(self._h, C.c_void_p(params.data_ptr()),
                                     C.c_void_p(feat.data_ptr()), n, C.c_void_p(y.data_ptr()),
                                     self._stream(stream))
        self._check(s, "rbf_mlp_forward")
        return y

    def mlp_train_step(self, params, m, v, step: int, lr: float, feat, target, idx=None,
                       n=None, grad=None, loss=None, stream=None):
        """One minibatch step (step 0: gradient only). idx: int32 CUDA tensor of sample rows."""
        n = int(idx.numel() if idx is not None else (n if n is not None else feat.shape[0]))
        ptr = lambda t: C.c_void_p(t.data_ptr() if t is not None else 0)  # noqa: E731
        s = self.lib.rbf_mlp_train_step(self._h, ptr(params), ptr(m), ptr(v), int(step),
                                        float(lr), ptr(feat), ptr(target), ptr(idx), n, ptr(grad),
                                        ptr(loss), self._stream(stream))
        self._check(s, "rbf_mlp_train_step")

    def warm_start(self, params, out=None, stream=None):
        """c0 = sigma * network(features) for every centre (caller order, float64)."""
        torch = _torch()
        c0 = out if out is not None else torch.empty(self.M, dtype=torch.float64,
                                                     device=f"cuda:{self.device}")
        s = self.lib.rbf_warm_start(self._h, C.c_void_p(params.data_ptr()),
                                    C.c_void_p(c0.data_ptr()), self._stream(stream))
        self._check(s, "rbf_warm_start")
        return c0

    def mlp_targets(self, c, out=None, stream=None):
        """The network's training targets t_j = c_j / sigma (caller order, float32)."""
        torch = _torch()
        t = out if out is not None else torch.empty(self.M, dtype=torch.float32, device=c.device)
        s = self.lib.rbf_mlp_targets(self._h, _dptr(c, "c"), C.c_void_p(t.data_ptr()),
                                     self._stream(stream))
        self._check(s, "rbf_mlp_targets")
        return t

    def autotune(self, stream=None):
        """Time the batched CG loop's launch configurations and keep the fastest."""
        self._check(self.lib.rbf_autotune(self._h, self._stream(stream)), "rbf_autotune")
        return self.tuning()

    def tuning(self):
        b, ch, nt, us = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        self._check(self.lib.rbf_get_tuning(self._h, C.byref(b), C.byref(ch), C.byref(nt),
                                            C.byref(us)), "rbf_get_tuning")
        return dict(spmv_blocks_per_sm=b.value, spmv_chunk=ch.value, update_threads=nt.value,
                    us_per_iteration=us.value)

    # -- diagnostics --------------------------------------------------------------------
    def layout(self):
        nv, vb, gx, gy = C.c_int64(), C.c_int(), C.c_int(), C.c_int()
        self._check(self.lib.rbf_get_layout(self._h, C.byref(nv), C.byref(vb), C.byref(gx),
                                            C.byref(gy)), "rbf_get_layout")
        return dict(nvals=nv.value, value_bytes=vb.value, gx=gx.value, gy=gy.value)

    def layout_stats(self, stream=None):
        """Stored values, nonzeros of the upper triangle (diagonal included), row groups,
        dropped Gram entries (always 0) and host blocks (0: B in device memory) of the last
        assembly."""
        st = _lib.LayoutStats()
        self._check(self.lib.rbf_get_layout_stats(self._h, C.byref(st), self._stream(stream)),
                    "rbf_get_layout_stats")
        return dict(stored_values=st.stored_values, nonzeros=st.nonzeros,
                    row_groups=st.row_groups, dropped=st.dropped, host_blocks=st.host_blocks)

    def set_param(self, name: str, value: float):
        """Context parameters: "inner_tol", "max_refinements", "store_a", "autotune",
        "spmv_blocks_per_sm", "spmv_chunk", "update_threads", "b_device_mb" (see
        include/rbf.h)."""
        self._check(self.lib.rbf_set_param(self._h, name.encode(), float(value)), "rbf_set_param")

    def launch_count(self) -> int:
        n = C.c_int64()
        self._check(self.lib.rbf_get_launch_count(self._h, C.byref(n)), "rbf_get_launch_count")
        return n.value

    def bench_spmv(self, reps: int, stream=None):
        """Launch the solver's SpMV kernel reps times (timing hook; needs a prior solve)."""
        self._check(self.lib.rbf_bench_spmv(self._h, int(reps), self._stream(stream)),
                    "rbf_bench_spmv")

    def bench_cg(self, reps: int, stream=None):
        """Run reps CG iterations as individual kernel launches (timing hook; needs a prior
        solve; overwrites the solver workspace)."""
        self._check(self.lib.rbf_bench_cg(self._h, int(reps), self._stream(stream)), "rbf_bench_cg")

    def bench_fma(self, prec: str, reps: int, stream=None) -> float:
        """Launch the FMA throughput probe in `prec` ("fp64" or "fp32_refine" for FP32);
        returns the flops it performs (timing hook)."""
        fl = C.c_double()
        self._check(self.lib.rbf_bench_fma(self._h, _lib.PRECS[prec], int(reps), C.byref(fl),
                                           self._stream(stream)), "rbf_bench_fma")
        return fl.value

    def bench_residual(self, reps: int, stream=None):
        """Run reps FP64 refinement residual passes at the current iterate (timing hook)."""
        self._check(self.lib.rbf_bench_residual(self._h, int(reps), self._stream(stream)),
                    "rbf_bench_residual")

    def bench_cg_loop(self, reps: int, stream=None):
        """Run reps CG iterations in the solver's own loop (persistent kernel or graph; timing
        hook; needs a prior solve; overwrites the solver workspace; synchronises)."""
        self._check(self.lib.rbf_bench_cg_loop(self._h, int(reps), self._stream(stream)),
                    "rbf_bench_cg_loop")

    def export_upper(self, stream=None):
        """The assembled upper triangle of B as COO (caller's centre indices), plus b and the
        support counts, as CUDA tensors."""
        torch = _torch()
        dev = f"cuda:{self.device}"
        cap = self.layout()["nvals"]
        row = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        col = torch.empty_like(row)
        val = torch.empty(max(cap, 1), dtype=torch.float64, device=dev)
        b = torch.empty(self.M, dtype=torch.float64, device=dev)
        sup = torch.empty(self.M, dtype=torch.int32, device=dev)
        nnz = C.c_int64()
        s = self.lib.rbf_export_upper(self._h, cap, C.c_void_p(row.data_ptr()),
                                      C.c_void_p(col.data_ptr()), C.c_void_p(val.data_ptr()),
                                      C.c_void_p(b.data_ptr()), C.c_void_p(sup.data_ptr()),
                                      C.byref(nnz), self._stream(stream))
        self._check(s, "rbf_export_upper")
        n = nnz.value
        return row[:n], col[:n], val[:n], b, sup


def pack_tiles(problems):
    """Concatenate per-tile host arrays. problems: sequence of (points (N,2), h (N,),
    centres (M,2), R, bbox). Returns (tiles, cx, cy, px, py, h) with numpy arrays."""
    import numpy as np
    tiles, C_, P_, H_ = [], [], [], []
    c0 = p0 = 0
    for pts, hh, cen, R, bbox in problems:
        pts = np.asarray(pts, dtype=np.float64).reshape(-1, 2)
        cen = np.asarray(cen, dtype=np.float64).reshape(-1, 2)
        tiles.append(dict(c0=c0, M=len(cen), p0=p0, N=len(pts), R=float(R), bbox=tuple(bbox)))
        c0 += len(cen)
        p0 += len(pts)
        C_.append(cen)
        P_.append(pts)
        H_.append(np.asarray(hh, dtype=np.float64).reshape(-1))
    Cc, Pp, Hh = np.concatenate(C_), np.concatenate(P_), np.concatenate(H_)
    return tiles, Cc[:, 0].copy(), Cc[:, 1].copy(), Pp[:, 0].copy(), Pp[:, 1].copy(), Hh


def fit_tiles(problems, kernel: str = "w31", prec: str = "fp32_refine", tol: float = 1e-10,
              maxit: int = 200000, min_support: int = 3, ctx: Context | None = None,
              device: int = 0):
    """Fit many independent tiles together. problems: as for pack_tiles. Returns
    (list of per-tile c on the device, info, per-tile info, ctx)."""
    torch = _torch()
    dev = f"cuda:{device}"
    tiles, cx, cy, px, py, hh = pack_tiles(problems)
    t = [torch.as_tensor(a).to(dev) for a in (cx, cy, px, py, hh)]
    ctx = ctx or Context(device)
    ctx.bin_tiles(tiles, *t)
    ctx.assemble(kernel, prec)
    c, info, tinfo = ctx.solve_tiles(tol=tol, maxit=maxit, min_support=min_support)
    cs = [c[d["c0"]:d["c0"] + d["M"]] for d in tiles]
    return cs, info, tinfo, ctx


def fit_windows(points, h, centres, R: float, wx: int, wy: int, overlap: float,
                kernel: str = "w31", prec: str = "fp32_refine", bbox=(0.0, 0.0, 1.0, 1.0),
                tol: float = 1e-10, maxit: int = 200000, min_support: int = 3,
                margin: float | None = None, ctx: Context | None = None, device: int = 0):
    """Moving-window fit: wx x wy overlapping windows fitted as one batch. Returns (c, info,
    per-window info, ctx); c holds the windows' weights one window after another
    (ctx.window_centres() maps them to input centres), ctx.eval_windows(_grid) blends them."""
    torch = _torch()
    dev = f"cuda:{device}"

    def dev64(a):
        t = a if isinstance(a, torch.Tensor) else torch.as_tensor(a)
        return t.to(device=dev, dtype=torch.float64)

    P, H, Cc = dev64(points), dev64(h), dev64(centres)
    ctx = ctx or Context(device)
    ctx.bin_windows(Cc[:, 0].contiguous(), Cc[:, 1].contiguous(), P[:, 0].contiguous(),
                    P[:, 1].contiguous(), H.contiguous(), R, bbox, wx, wy, overlap, margin)
    ctx.assemble(kernel, prec)
    c, info, tinfo = ctx.solve_tiles(tol=tol, maxit=maxit, min_support=min_support)
    return c, info, tinfo, ctx


def fit(points, h, centres, R: float, kernel: str = "w31", prec: str = "fp64",
        bbox=(0.0, 0.0, 1.0, 1.0), tol: float = 1e-10, maxit: int = 200000, min_support: int = 3,
        c0=None, ctx: Context | None = None, device: int = 0):
    """Whole fit. points (N,2), h (N,), centres (M,2): torch tensors or numpy arrays (host
    inputs are copied to the device). Returns (c on the device, info dict, ctx)."""
    torch = _torch()
    dev = f"cuda:{device}"

    def dev64(a):
        t = a if isinstance(a, torch.Tensor) else torch.as_tensor(a)
        return t.to(device=dev, dtype=torch.float64, non_blocking=True)

    P, H, Cc = dev64(points), dev64(h), dev64(centres)
    ctx = ctx or Context(device)
    ctx.bin(Cc[:, 0].contiguous(), Cc[:, 1].contiguous(), P[:, 0].contiguous(),
            P[:, 1].contiguous(), H.contiguous(), R, bbox)
    ctx.assemble(kernel, prec)
    c, info = ctx.solve(tol=tol, maxit=maxit, min_support=min_support,
                        c0=None if c0 is None else dev64(c0))
    return c, info, ctx


def fit_poly(points, h, centres, R: float, kernel: str = "w31", prec: str = "fp64",
             bbox=(0.0, 0.0, 1.0, 1.0), tol: float = 1e-10, maxit: int = 200000,
             min_support: int = 3, ctx: Context | None = None, device: int = 0):
    """Whole fit with linear polynomial reproduction (Eq. 10). Returns (c, k, info, ctx) with
    c and k = (a_x, a_y, a_0) on the device."""
    torch = _torch()
    dev = f"cuda:{device}"

    def dev64(a):
        t = a if isinstance(a, torch.Tensor) else torch.as_tensor(a)
        return t.to(device=dev, dtype=torch.float64, non_blocking=True)

    P, H, Cc = dev64(points), dev64(h), dev64(centres)
    ctx = ctx or Context(device)
    ctx.bin(Cc[:, 0].contiguous(), Cc[:, 1].contiguous(), P[:, 0].contiguous(),
            P[:, 1].contiguous(), H.contiguous(), R, bbox)
    ctx.assemble_poly(kernel, prec)
    c, k, info = ctx.solve_poly(tol=tol, maxit=maxit, min_support=min_support)
    return c, k, info, ctx
