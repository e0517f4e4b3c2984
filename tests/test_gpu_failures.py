"""Failure paths of the C-ABI, provoked from the host (no GPU fault, trap or hang):

* a non-finite start vector makes the CG step scalars non-finite: rbf_solve returns
  RBF_ERR_BREAKDOWN (FP64 and FP32 + refinement) and the context stays usable;
* a workspace allocator that returns NULL makes the call that needed the memory return
  RBF_ERR_ALLOC with a message; with room again the same context completes the fit;
* an allocator with no room for the stored values of A keeps the matrix-free residual and
  still reaches the oracle's surface;
* a grid-barrier wait of the persistent CG kernel that runs out (a barrier told to wait for a
  block that does not exist) returns RBF_ERR_TIMEOUT and leaves the context usable."""
import ctypes as C

import numpy as np
import pytest

import datagen as dg
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1806_07884_gb300 as pkg  # noqa: E402
from paper_1806_07884_gb300 import _lib  # noqa: E402

FP64_BAR = 1e-9
MIXED_BAR = 1e-6


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _binned(pb, prec):
    ctx = pkg.Context()
    ctx.bin(_dev(pb.centres[:, 0]), _dev(pb.centres[:, 1]), _dev(pb.points[:, 0]),
            _dev(pb.points[:, 1]), _dev(pb.h), pb.R)
    ctx.assemble(pb.kernel, prec)
    return ctx


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_start_vector_is_a_breakdown(prec, bad):
    pb = dg.config_franke(seed=21, N=4000, M=400)
    c_ref, _ = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    ctx = _binned(pb, prec)
    c0 = np.zeros(pb.M)
    c0[17] = bad
    c, info = ctx.solve(tol=1e-13, c0=_dev(c0), raise_on_fail=False)
    assert info["status"] == _lib.RBF_ERR_BREAKDOWN, info
    assert "breakdown" in ctx.lib.rbf_last_error(ctx._h).decode().lower()
    # the context is still usable: a cold solve on it reaches the oracle's weights
    c, info = ctx.solve(tol=1e-13)
    assert info["status"] == 0
    f = O.evaluate(c.cpu().numpy(), pb.centres, pb.points, pb.R, pb.kernel)
    f_ref = O.evaluate(c_ref, pb.centres, pb.points, pb.R, pb.kernel)
    assert O.rel_err(f, f_ref) <= (FP64_BAR if info["promoted"] or prec == "fp64" else MIXED_BAR)
    ctx.close()


class _BudgetAllocator:
    """Workspace allocator over torch's caching allocator that refuses (returns NULL) any
    request larger than `limit` bytes, and every request once `fail_all` is set."""

    def __init__(self, limit=1 << 62):
        self.limit, self.fail_all, self.refused = limit, False, 0

        def alloc(nbytes, stream, user):
            if self.fail_all or nbytes > self.limit:
                self.refused += 1
                return None
            return torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))

        def free(ptr, nbytes, stream, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc_fn = _lib.ALLOC_FN(alloc)
        self.free_fn = _lib.FREE_FN(free)


def _raw_context(a):
    lib = _lib.load()
    h = C.c_void_p()
    assert lib.rbf_create(C.byref(h), 0, a.alloc_fn, a.free_fn, None) == 0
    return lib, h


def _bin(lib, h, pb, keep):
    cx, cy, px, py, hh = (_dev(pb.centres[:, 0]), _dev(pb.centres[:, 1]), _dev(pb.points[:, 0]),
                          _dev(pb.points[:, 1]), _dev(pb.h))
    keep += [cx, cy, px, py, hh]
    box = (C.c_double * 4)(*pb.bbox)
    return lib.rbf_bin(h, cx.data_ptr(), cy.data_ptr(), pb.M, px.data_ptr(), py.data_ptr(),
                       hh.data_ptr(), pb.N, pb.R, box, None)


def test_allocator_returning_null_is_reported_and_recoverable():
    pb = dg.config_franke(seed=22, N=6000, M=600)
    a = _BudgetAllocator()
    lib, h = _raw_context(a)
    keep = []
    a.fail_all = True
    assert _bin(lib, h, pb, keep) == _lib.RBF_ERR_ALLOC
    assert b"allocation" in lib.rbf_last_error(h)
    assert a.refused >= 1
    # room again: the same context bins; then no room for B: the assembly reports it
    a.fail_all = False
    assert _bin(lib, h, pb, keep) == 0
    nvals = C.c_int64()
    assert lib.rbf_get_layout(h, C.byref(nvals), None, None, None) == 0
    a.limit = 8 * nvals.value - 1                 # the FP64 values of B do not fit
    assert lib.rbf_assemble(h, _lib.KERNELS[pb.kernel], _lib.PRECS["fp64"], None) == \
        _lib.RBF_ERR_ALLOC
    # a solve before a successful assembly is an argument error, not a crash
    c = torch.zeros(pb.M, dtype=torch.float64, device="cuda")
    info = _lib.SolveInfo()
    assert lib.rbf_solve(h, c.data_ptr(), 0, 1e-13, 10000, 3, C.byref(info), None) != 0
    # room again: assembly and solve on the same context reach the oracle
    a.limit = 1 << 62
    assert lib.rbf_assemble(h, _lib.KERNELS[pb.kernel], _lib.PRECS["fp64"], None) == 0
    assert lib.rbf_solve(h, c.data_ptr(), 0, 1e-13, 10000, 3, C.byref(info), None) == 0
    c_ref, _ = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    assert O.rel_err(c.cpu().numpy(), c_ref) <= FP64_BAR
    assert lib.rbf_destroy(h) == 0


def test_no_room_for_stored_a_keeps_the_matrix_free_residual():
    pb = dg.config_franke(seed=23, N=6000, M=600)
    a = _BudgetAllocator()
    lib, h = _raw_context(a)
    keep = []
    assert _bin(lib, h, pb, keep) == 0
    # the stored values of A take about 8 B x N x 9 x centres per cell: far more than B
    nvals = C.c_int64()
    lib.rbf_get_layout(h, C.byref(nvals), None, None, None)
    a.limit = max(16 * nvals.value, 64 * pb.M * 8)
    assert 8 * pb.N * 9 * 6 > a.limit
    assert lib.rbf_assemble(h, _lib.KERNELS[pb.kernel], _lib.PRECS["fp32_refine"], None) == 0
    assert a.refused >= 1
    c = torch.zeros(pb.M, dtype=torch.float64, device="cuda")
    info = _lib.SolveInfo()
    assert lib.rbf_solve(h, c.data_ptr(), 0, 1e-12, 10000, 3, C.byref(info), None) == 0
    c_ref, _ = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    f = O.evaluate(c.cpu().numpy(), pb.centres, pb.points, pb.R, pb.kernel)
    f_ref = O.evaluate(c_ref, pb.centres, pb.points, pb.R, pb.kernel)
    assert O.rel_err(f, f_ref) <= MIXED_BAR
    assert lib.rbf_destroy(h) == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_barrier_wait_that_runs_out_is_a_timeout(prec):
    """The persistent solve's grid barriers are told to wait for one block more than the grid
    has (the "cg_barrier_test" hook): every wait runs out after its 2 s limit, every block
    leaves, rbf_solve returns RBF_ERR_TIMEOUT, and the same context then completes the fit."""
    pb = dg.config_franke(seed=22, N=4000, M=400)
    c_ref, _ = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    ctx = _binned(pb, prec)
    ctx.set_param("cg_persistent", 1)
    ctx.set_param("cg_barrier_test", 1)
    with pytest.raises(pkg.RBFError) as e:
        ctx.solve(tol=1e-13)
    assert "RBF_ERR_TIMEOUT" in str(e.value)
    ctx.set_param("cg_barrier_test", 0)
    c, info = ctx.solve(tol=1e-13)
    assert info["status"] == 0
    f = O.evaluate(c.cpu().numpy(), pb.centres, pb.points, pb.R, pb.kernel)
    f_ref = O.evaluate(c_ref, pb.centres, pb.points, pb.R, pb.kernel)
    assert O.rel_err(f, f_ref) <= (FP64_BAR if prec == "fp64" else MIXED_BAR)
    ctx.close()
