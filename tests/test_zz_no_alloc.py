"""rbf_eval_noalloc -- evaluation for callers that cannot allocate device memory -- agrees
with rbf_eval on two calls in a row (different centres, coefficients and queries), calling
both through the C-ABI. Collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import datagen as dg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1806_07884_gb300 as pkg  # noqa: E402
from paper_1806_07884_gb300 import _lib  # noqa: E402

FP64_BAR = 1e-9


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _case(seed, M, Q, kind):
    pb = dg.config_small(seed, 4 * M, M, K=20.0, kernel=kind)
    rng = np.random.default_rng(seed + 100)
    c = rng.standard_normal(M)
    q = rng.random((Q, 2)) * 1.1 - 0.05          # some queries outside the box
    return pb, c, q


def test_noalloc_eval_matches_context_eval_twice():
    lib = _lib.load()
    box = (ctypes.c_double * 4)(0.0, 0.0, 1.0, 1.0)
    for call, (seed, M, Q, kind) in enumerate([(1, 3000, 20000, "w31"), (2, 777, 5001, "w33")]):
        pb, c, q = _case(seed, M, Q, kind)
        C, c_d = _dev(pb.centres), _dev(c)
        cx, cy = C[:, 0].contiguous(), C[:, 1].contiguous()
        qx, qy = _dev(q[:, 0]), _dev(q[:, 1])
        # reference: the context path (rbf_bin / rbf_assemble / rbf_eval)
        ctx = pkg.Context()
        P = _dev(pb.points)
        ctx.bin(cx, cy, P[:, 0].contiguous(), P[:, 1].contiguous(), _dev(pb.h), pb.R)
        ctx.assemble(kind, "fp64")
        f_ref = ctx.eval(c_d, qx, qy).cpu().numpy()
        ctx.close()
        f = torch.full((Q,), np.nan, dtype=torch.float64, device="cuda")
        st = lib.rbf_eval_noalloc(cx.data_ptr(), cy.data_ptr(), c_d.data_ptr(), M, pb.R, box,
                                  _lib.KERNELS[kind], qx.data_ptr(), qy.data_ptr(), Q,
                                  f.data_ptr(), None)
        assert st == 0, (call, st)
        torch.cuda.synchronize()
        f = f.cpu().numpy()
        assert np.all(np.isfinite(f))
        err = np.max(np.abs(f - f_ref)) / max(np.max(np.abs(f_ref)), 1e-300)
        assert err <= FP64_BAR, (call, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = _lib.load()
    box = (ctypes.c_double * 4)(0.0, 0.0, 1.0, 1.0)
    x = torch.zeros(70000, dtype=torch.float64, device="cuda")
    # too many centres
    assert lib.rbf_eval_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 70000, 0.1, box, 1,
                                x.data_ptr(), x.data_ptr(), 1, x.data_ptr(), None) == _lib.RBF_ERR_LIMIT
    # too many cells (R too small for the box)
    assert lib.rbf_eval_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 10, 1e-3, box, 1,
                                x.data_ptr(), x.data_ptr(), 1, x.data_ptr(), None) == _lib.RBF_ERR_LIMIT
