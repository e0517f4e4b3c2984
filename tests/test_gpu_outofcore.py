"""B beyond device memory (Section 5, Eq. 13-16: the LSE matrix assembled block by block): with
the context parameter "b_device_mb" the stored values of B live in pinned, device-mapped host
memory, are assembled on the device in blocks of cell rows that fit the bound, and are read by
the solver over the host link.

Bars: the exported B (pattern exact, values to 1e-12 in FP64 and FP32 rounding in FP32), b
and the support counts equal those of the in-device assembly and of the oracle; the fits meet
the parity bars of the in-device path (FP64: c to max(1e-9, 1e-14 kappa); FP32 + FP64
refinement: f to 1e-6); the block count follows the bound."""
import numpy as np
import pytest
import scipy.sparse

import datagen as dg
import oracle as O
from oracle import poly_oracle as PO

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1806_07884_gb300 as pkg  # noqa: E402

FP64_BAR = 1e-9
MIXED_BAR = 1e-6


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _ctx(pb, b_device_mb, kind=None, prec="fp64", poly=False):
    ctx = pkg.Context()
    ctx.set_param("b_device_mb", b_device_mb)
    C, P = pb.centres, pb.points
    ctx.bin(_dev(C[:, 0]), _dev(C[:, 1]), _dev(P[:, 0]), _dev(P[:, 1]), _dev(pb.h), pb.R, pb.bbox)
    (ctx.assemble_poly if poly else ctx.assemble)(kind or pb.kernel, prec)
    return ctx


def _upper(ctx):
    row, col, val, b, sup = [t.cpu().numpy() for t in ctx.export_upper()]
    got = {}
    for i, j, v in zip(row, col, val):
        i, j = (int(i), int(j)) if i <= j else (int(j), int(i))
        got[(i, j)] = got.get((i, j), 0.0) + float(v)
    return got, b, sup


def _kappa(info_ref):
    free = ~info_ref["pinned"]
    B = info_ref["B"].toarray()[free][:, free]
    d = np.sqrt(np.diag(B))
    ev = np.linalg.eigvalsh(B / d[:, None] / d[None, :])
    return float(ev[-1] / ev[0])


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("mb", [0.05, 1e-6])
def test_host_b_equals_device_b_and_oracle(prec, mb):
    """Several blocks of cell rows (0.05 MB) and one cell row per block (1e-6 MB: below any
    row's size) give the in-device B, b and support counts."""
    pb = dg.config_terrain(seed=41, N=20000, M=2000)
    dctx = _ctx(pb, 0.0, prec=prec)
    hctx = _ctx(pb, mb, prec=prec)
    st_d, st_h = dctx.layout_stats(), hctx.layout_stats()
    assert st_d["host_blocks"] == 0
    assert st_h["host_blocks"] > 1
    assert st_h["stored_values"] == st_d["stored_values"]
    assert st_h["nonzeros"] == st_d["nonzeros"] and st_h["dropped"] == 0
    gd, bd, sd = _upper(dctx)
    gh, bh, sh = _upper(hctx)
    assert set(gd) == set(gh)
    scale = max(abs(v) for v in gd.values())
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert max(abs(gd[k] - gh[k]) for k in gd) <= tol * scale
    np.testing.assert_array_equal(sd, sh)
    assert O.rel_err(bh, bd) <= 1e-12
    A = O.design_matrix(pb.points, pb.centres, pb.R, pb.kernel)
    B, bref = O.normal_system(A, pb.h)
    Bu = scipy.sparse.triu(B).tocoo()
    ref = {(int(i), int(j)): v for i, j, v in zip(Bu.row, Bu.col, Bu.data) if v != 0.0}
    assert set(gh) == set(ref)
    assert max(abs(gh[k] - ref[k]) for k in ref) <= tol * scale
    assert O.rel_err(bh, bref) <= 1e-12
    np.testing.assert_array_equal(sh, O.support_counts(A))
    dctx.close()
    hctx.close()


@pytest.mark.parametrize("case", ["terrain", "clustered"])
def test_fit_with_host_b_matches_oracle(case):
    pb = (dg.config_terrain(seed=42, N=20000, M=2000) if case == "terrain"
          else dg.config_small(43, 6000, 400, clustered=True))
    c_ref, info_ref = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel, method="cholesky")
    f_ref = O.evaluate_grid(c_ref, pb.centres, pb.R, pb.kernel, 65)
    ctx = pkg.Context()
    ctx.set_param("b_device_mb", 0.02)
    c, info, ctx = pkg.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel, prec="fp64", tol=1e-14,
                           bbox=pb.bbox, ctx=ctx)
    assert ctx.layout_stats()["host_blocks"] > 1
    assert info["pinned"] == int(info_ref["pinned"].sum())
    assert O.rel_err(c.cpu().numpy(), c_ref) <= max(FP64_BAR, 1e-14 * _kappa(info_ref))
    assert O.rel_err(ctx.eval_grid(c, 65, 65, pb.bbox).cpu().numpy(), f_ref) <= FP64_BAR
    # the same context, FP32 B in host memory with FP64 refinement
    ctx.assemble(pb.kernel, "fp32_refine")
    assert ctx.layout_stats()["host_blocks"] > 1
    c32, info32 = ctx.solve(tol=1e-10)
    assert info32["refinements"] >= 1
    assert O.rel_err(ctx.eval_grid(c32, 65, 65, pb.bbox).cpu().numpy(), f_ref) <= MIXED_BAR
    # back to device memory: the host copy is dropped and the fit is unchanged
    ctx.set_param("b_device_mb", 0.0)
    ctx.assemble(pb.kernel, "fp64")
    assert ctx.layout_stats()["host_blocks"] == 0
    c2, _ = ctx.solve(tol=1e-14)
    assert O.rel_err(c2.cpu().numpy(), c_ref) <= max(FP64_BAR, 1e-14 * _kappa(info_ref))
    ctx.close()


def test_poly_fit_with_host_b_matches_oracle():
    pb = dg.config_franke(seed=44, N=5000, M=500)
    c_ref, k_ref, _ = PO.fit_poly(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    for prec, bar in (("fp64", FP64_BAR), ("fp32_refine", MIXED_BAR)):
        ctx = _ctx(pb, 0.01, prec=prec, poly=True)
        assert ctx.layout_stats()["host_blocks"] > 1
        c, k, info = ctx.solve_poly(tol=1e-13 if prec == "fp64" else 1e-12)
        f = ctx.eval_poly(c, k, _dev(pb.points[:, 0]), _dev(pb.points[:, 1])).cpu().numpy()
        f_ref = PO.evaluate_poly(c_ref, k_ref, pb.centres, pb.points, pb.R, pb.kernel)
        assert O.rel_err(f, f_ref) <= bar, prec
        ctx.close()


def test_b_device_mb_argument_range():
    ctx = pkg.Context()
    for bad in (-1.0, float("nan"), 2e9):
        with pytest.raises(pkg.RBFError) as e:
            ctx.set_param("b_device_mb", bad)
        assert "RBF_ERR_ARG" in str(e.value)
    ctx.set_param("b_device_mb", 0.0)
    ctx.close()
