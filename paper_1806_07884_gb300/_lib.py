"""ctypes binding of librbf (include/rbf.h): loads the in-tree shared library and
declares the C signatures. Argument marshalling only -- all work runs in the CUDA
kernels of the library. There is no fallback: a missing library is an error."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librbf.so")

RBF_OK, RBF_ERR_ARG, RBF_ERR_ALLOC, RBF_ERR_CUDA, RBF_ERR_NOT_CONVERGED, RBF_ERR_BREAKDOWN, \
    RBF_ERR_LIMIT, RBF_ERR_TIMEOUT = range(8)
STATUS_NAMES = {0: "RBF_OK", 1: "RBF_ERR_ARG", 2: "RBF_ERR_ALLOC", 3: "RBF_ERR_CUDA",
                4: "RBF_ERR_NOT_CONVERGED", 5: "RBF_ERR_BREAKDOWN", 6: "RBF_ERR_LIMIT",
                7: "RBF_ERR_TIMEOUT"}
KERNELS = {"w30": 0, "w31": 1, "w32": 2, "w33": 3}
PRECS = {"fp64": 0, "fp32_refine": 1}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int),
                ("rel_residual", C.c_double), ("pinned", C.c_int64), ("promoted", C.c_int)]


class Tile(C.Structure):
    _fields_ = [("c0", C.c_int64), ("M", C.c_int64), ("p0", C.c_int64), ("N", C.c_int64),
                ("R", C.c_double), ("bbox", C.c_double * 4)]


class TileInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int),
                ("rel_residual", C.c_double), ("pinned", C.c_int64), ("status", C.c_int),
                ("promoted", C.c_int)]


class LayoutStats(C.Structure):
    _fields_ = [("stored_values", C.c_int64), ("nonzeros", C.c_int64),
                ("row_groups", C.c_int64), ("dropped", C.c_int64), ("host_blocks", C.c_int64)]


_P = C.c_void_p
_D = C.c_double
_I = C.c_int
_I64 = C.c_int64

# name -> (restype, argtypes); mirrors include/rbf.h
SIGNATURES = {
    "rbf_create": (_I, [C.POINTER(_P), _I, ALLOC_FN, FREE_FN, _P]),
    "rbf_destroy": (_I, [_P]),
    "rbf_last_error": (C.c_char_p, [_P]),
    "rbf_bin": (_I, [_P, _P, _P, _I64, _P, _P, _P, _I64, _D, C.POINTER(_D), _P]),
    "rbf_max_candidates": (_I, []),
    "rbf_assemble": (_I, [_P, _I, _I, _P]),
    "rbf_solve": (_I, [_P, _P, _I, _D, _I, _I, C.POINTER(SolveInfo), _P]),
    "rbf_eval": (_I, [_P, _P, _P, _P, _I64, _P, _P]),
    "rbf_eval_grid": (_I, [_P, _P, _I, _I, C.POINTER(_D), _P, _P]),
    "rbf_get_layout": (_I, [_P, C.POINTER(_I64), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "rbf_get_layout_stats": (_I, [_P, C.POINTER(LayoutStats), _P]),
    "rbf_assemble_poly": (_I, [_P, _I, _I, _P]),
    "rbf_solve_poly": (_I, [_P, _P, _P, _D, _I, _I, C.POINTER(SolveInfo), _P]),
    "rbf_eval_poly": (_I, [_P, _P, _P, _P, _P, _I64, _P, _P]),
    "rbf_eval_grid_poly": (_I, [_P, _P, _P, _I, _I, C.POINTER(_D), _P, _P]),
    "rbf_export_upper": (_I, [_P, _I64, _P, _P, _P, _P, _P, C.POINTER(_I64), _P]),
    "rbf_get_launch_count": (_I, [_P, C.POINTER(_I64)]),
    "rbf_set_param": (_I, [_P, C.c_char_p, _D]),
    "rbf_selftest_sqrt": (_I, [_P, _P, _I64, _P]),
    "rbf_eval_noalloc": (_I, [_P, _P, _P, _I64, _D, C.POINTER(_D), _I, _P, _P, _I64, _P, _P]),
    "rbf_bench_spmv": (_I, [_P, _I, _P]),
    "rbf_bench_cg": (_I, [_P, _I, _P]),
    "rbf_bench_cg_loop": (_I, [_P, _I, _P]),
    "rbf_bench_fma": (_I, [_P, _I, _I64, C.POINTER(_D), _P]),
    "rbf_bench_residual": (_I, [_P, _I, _P]),
    "rbf_bin_tiles": (_I, [_P, C.POINTER(Tile), _I, _P, _P, _I64, _P, _P, _P, _I64, _P]),
    "rbf_solve_tiles": (_I, [_P, _P, _I, _D, _I, _I, C.POINTER(TileInfo), C.POINTER(SolveInfo), _P]),
    "rbf_autotune": (_I, [_P, _P]),
    "rbf_eval_tiles": (_I, [_P, _P, _P, _P, C.POINTER(_I64), _P, _P]),
    "rbf_eval_tiles_grid": (_I, [_P, _P, _I, _I, _P, _P]),
    "rbf_bin_windows": (_I, [_P, _P, _P, _I64, _P, _P, _P, _I64, _D, C.POINTER(_D), _I, _I, _D, _D,
                             _P]),
    "rbf_window_sizes": (_I, [_P, C.POINTER(_I64), C.POINTER(_I64)]),
    "rbf_window_centres": (_I, [_P, _P, _I64, _P]),
    "rbf_eval_windows": (_I, [_P, _P, _P, _P, _I64, _P, _P]),
    "rbf_eval_windows_grid": (_I, [_P, _P, _I, _I, C.POINTER(_D), _P, _P]),
    "rbf_features": (_I, [_P, _P, _P, _P]),
    "rbf_mlp_forward": (_I, [_P, _P, _P, _I64, _P, _P]),
    "rbf_mlp_train_step": (_I, [_P, _P, _P, _P, _I, _D, _P, _P, _P, _I64, _P, _P, _P]),
    "rbf_warm_start": (_I, [_P, _P, _P, _P]),
    "rbf_mlp_targets": (_I, [_P, _P, _P, _P]),
    "rbf_get_tuning": (_I, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(_D)]),
}

_lib = None


class RBFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load librbf.so (built by __graft_entry__.build() / paper_1806_07884_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
