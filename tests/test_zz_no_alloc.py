"""rbf_eval_noalloc -- evaluation for callers that cannot allocate device memory -- called
through the C-ABI: it agrees with rbf_eval (the context path) and with the oracle's Eq. 3
on two calls in a row (different centres, coefficients and queries), with centres outside
the bounding box, at its size limits, and when two calls are queued on one non-default
stream. Collected last so that a run stopping at the first failure has already run every
other test."""
import ctypes

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
LIMIT = 65536          # largest M and largest cell count the static scratch accepts


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _case(seed, M, Q, kind):
    pb = dg.config_small(seed, 4 * M, M, K=20.0, kernel=kind)
    rng = np.random.default_rng(seed + 100)
    c = rng.standard_normal(M)
    q = rng.random((Q, 2)) * 1.1 - 0.05          # some queries outside the box
    return pb, c, q


def _noalloc(lib, C, c, q, R, kind, box=(0.0, 0.0, 1.0, 1.0), stream=None, out=None):
    """Queue one rbf_eval_noalloc call; returns the device output (not synchronised)."""
    cx, cy = _dev(C[:, 0]), _dev(C[:, 1])
    c_d, qx, qy = _dev(c), _dev(q[:, 0]), _dev(q[:, 1])
    f = out if out is not None else torch.full((q.shape[0],), np.nan, dtype=torch.float64,
                                               device="cuda")
    b = (ctypes.c_double * 4)(*box)
    st = lib.rbf_eval_noalloc(cx.data_ptr(), cy.data_ptr(), c_d.data_ptr(), C.shape[0], R, b,
                              _lib.KERNELS[kind], qx.data_ptr(), qy.data_ptr(), q.shape[0],
                              f.data_ptr(), stream)
    assert st == 0, st
    return f, (cx, cy, c_d, qx, qy)        # the inputs stay alive until the caller syncs


def test_noalloc_eval_matches_context_eval_twice():
    lib = _lib.load()
    for call, (seed, M, Q, kind) in enumerate([(1, 3000, 20000, "w31"), (2, 777, 5001, "w33")]):
        pb, c, q = _case(seed, M, Q, kind)
        C, c_d = _dev(pb.centres), _dev(c)
        cx, cy = C[:, 0].contiguous(), C[:, 1].contiguous()
        qx, qy = _dev(q[:, 0]), _dev(q[:, 1])
        # the existing entry point: the context path (rbf_bin / rbf_assemble / rbf_eval)
        ctx = pkg.Context()
        P = _dev(pb.points)
        ctx.bin(cx, cy, P[:, 0].contiguous(), P[:, 1].contiguous(), _dev(pb.h), pb.R)
        ctx.assemble(kind, "fp64")
        f_ctx = ctx.eval(c_d, qx, qy).cpu().numpy()
        ctx.close()
        f, keep = _noalloc(lib, pb.centres, c, q, pb.R, kind)
        torch.cuda.synchronize()
        f = f.cpu().numpy()
        assert np.all(np.isfinite(f))
        err = np.max(np.abs(f - f_ctx)) / max(np.max(np.abs(f_ctx)), 1e-300)
        assert err <= FP64_BAR, (call, err)
        # and Eq. 3 itself, as the oracle evaluates it
        f_or = O.evaluate(c, pb.centres, q, pb.R, kind)
        assert O.rel_err(f, f_or) <= FP64_BAR, (call, O.rel_err(f, f_or))


def test_noalloc_centres_outside_the_box():
    """Centres just outside bbox are clamped into the edge cells; every pair within R of a
    query is still found."""
    lib = _lib.load()
    rng = np.random.default_rng(11)
    M, Q, kind = 1500, 8000, "w31"
    C = rng.random((M, 2)) * 1.06 - 0.03            # about 12% of the centres outside [0, 1]^2
    R = dg.support_radius(M, 20.0)
    c = rng.standard_normal(M)
    q = rng.random((Q, 2)) * 1.1 - 0.05
    f, keep = _noalloc(lib, C, c, q, R, kind)
    torch.cuda.synchronize()
    f_or = O.evaluate(c, C, q, R, kind)
    assert O.rel_err(f.cpu().numpy(), f_or) <= FP64_BAR


def test_noalloc_at_its_limits():
    """M = 65536 centres on a grid of exactly 65536 cells (256 x 256): the last cell's start
    is written at the end of its region."""
    lib = _lib.load()
    rng = np.random.default_rng(12)
    R = 1.0 / 255.5            # cell side R (1 + 2^-30): ceil(1 / side) = 256 cells per axis
    C = rng.random((LIMIT, 2))
    c = rng.standard_normal(LIMIT)
    q = rng.random((30000, 2))
    f, keep = _noalloc(lib, C, c, q, R, "w30")
    torch.cuda.synchronize()
    f_or = O.evaluate(c, C, q, R, "w30")
    assert O.rel_err(f.cpu().numpy(), f_or) <= FP64_BAR


def test_noalloc_two_calls_on_one_stream():
    """Two calls queued back to back on one non-default stream, one synchronisation at the
    end: the second call's binning waits for the first call's evaluation."""
    lib = _lib.load()
    s = torch.cuda.Stream()
    pa, ca, qa = _case(3, 2000, 12000, "w31")
    pb, cb, qb = _case(4, 900, 7000, "w33")
    with torch.cuda.stream(s):
        fa, ka = _noalloc(lib, pa.centres, ca, qa, pa.R, "w31", stream=s.cuda_stream)
        fb, kb = _noalloc(lib, pb.centres, cb, qb, pb.R, "w33", stream=s.cuda_stream)
    s.synchronize()
    assert O.rel_err(fa.cpu().numpy(), O.evaluate(ca, pa.centres, qa, pa.R, "w31")) <= FP64_BAR
    assert O.rel_err(fb.cpu().numpy(), O.evaluate(cb, pb.centres, qb, pb.R, "w33")) <= FP64_BAR


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = _lib.load()
    box = (ctypes.c_double * 4)(0.0, 0.0, 1.0, 1.0)
    x = torch.zeros(70000, dtype=torch.float64, device="cuda")
    # too many centres
    assert lib.rbf_eval_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), LIMIT + 1, 0.1, box, 1,
                                x.data_ptr(), x.data_ptr(), 1, x.data_ptr(), None) == _lib.RBF_ERR_LIMIT
    # too many cells: 257 x 256 (R too small for the box)
    wide = (ctypes.c_double * 4)(0.0, 0.0, 256.5 / 255.5, 1.0)
    assert lib.rbf_eval_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 10, 1.0 / 255.5, wide,
                                1, x.data_ptr(), x.data_ptr(), 1, x.data_ptr(),
                                None) == _lib.RBF_ERR_LIMIT
    assert lib.rbf_eval_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 10, 1e-3, box, 1,
                                x.data_ptr(), x.data_ptr(), 1, x.data_ptr(), None) == _lib.RBF_ERR_LIMIT
