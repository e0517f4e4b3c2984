"""GPU parity of the fit with linear polynomial reproduction (Section 3, Eq. 6-10) through the
C-ABI (rbf_assemble_poly / rbf_solve_poly / rbf_eval_poly / rbf_eval_grid_poly) against the
oracle's bordered least-squares solution (oracle/poly_oracle.py).

Bars as for the fit without the polynomial: FP64 path c and k to max(1e-9, 1e-14 kappa)
(kappa: condition number of the Jacobi-scaled bordered matrix), the surface at the data points
and on a grid to 1e-9; FP32 + FP64 refinement: the surface to 1e-6. Linear data are reproduced
exactly (c = 0, k = the data's coefficients). Table 4's synthetic errors with the linear
polynomial are reproduced through the GPU path."""
import os

import numpy as np
import pytest

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


def _case(name):
    if name == "franke":
        return dg.config_franke(seed=31, N=5000, M=500)
    if name == "terrain":
        return dg.config_terrain(seed=32, N=20000, M=2000)
    if name == "clustered":
        return dg.config_small(33, 6000, 400, clustered=True)
    raise KeyError(name)


def _kappa(K, pin):
    keep = np.concatenate([np.nonzero(~pin)[0], K.shape[0] - 3 + np.arange(3)])
    Kd = K[keep][:, keep].toarray()
    d = 1.0 / np.sqrt(np.diag(Kd))
    ev = np.linalg.eigvalsh(Kd * d[:, None] * d[None, :])
    return ev[-1] / ev[0]


def _fit(pb, kind, prec, tol, min_support=3, bbox=None):
    c, k, info, ctx = pkg.fit_poly(pb.points, pb.h, pb.centres, pb.R, kind, prec=prec, tol=tol,
                                   min_support=min_support, bbox=bbox or pb.bbox)
    return c, k, info, ctx


@pytest.mark.parametrize("case,kind", [("franke", "w31"), ("terrain", "w31"), ("clustered", "w31"),
                                       ("franke", "w33"), ("franke", "w30")])
def test_poly_fp64_matches_oracle(case, kind):
    pb = _case(case)
    c_ref, k_ref, d = PO.fit_poly(pb.points, pb.h, pb.centres, pb.R, kind)
    c, k, info, ctx = _fit(pb, kind, "fp64", 1e-14)
    c, k = c.cpu().numpy(), k.cpu().numpy()
    assert info["status"] == 0, info
    assert info["pinned"] == int(d["pinned"].sum())
    bar = max(FP64_BAR, 1e-14 * _kappa(d["K"], d["pinned"]))
    ref = np.concatenate([c_ref, k_ref])
    assert np.abs(np.concatenate([c, k]) - ref).max() <= bar * np.abs(ref).max()
    f = ctx.eval_poly(_dev(c), _dev(k), _dev(pb.points[:, 0]), _dev(pb.points[:, 1])).cpu().numpy()
    f_ref = PO.evaluate_poly(c_ref, k_ref, pb.centres, pb.points, pb.R, kind)
    assert O.rel_err(f, f_ref) <= FP64_BAR
    n = 41
    g = ctx.eval_grid_poly(_dev(c), _dev(k), n, n, pb.bbox).cpu().numpy()
    gx = np.linspace(pb.bbox[0], pb.bbox[2], n)
    gy = np.linspace(pb.bbox[1], pb.bbox[3], n)
    X, Y = np.meshgrid(gx, gy)
    g_ref = PO.evaluate_poly(c_ref, k_ref, pb.centres, np.stack([X.ravel(), Y.ravel()], 1), pb.R,
                             kind).reshape(n, n)
    assert O.rel_err(g, g_ref) <= FP64_BAR
    ctx.close()


@pytest.mark.parametrize("case", ["franke", "terrain", "clustered"])
def test_poly_fp32_refine_surface_matches_oracle(case):
    pb = _case(case)
    c_ref, k_ref, _ = PO.fit_poly(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    c, k, info, ctx = _fit(pb, pb.kernel, "fp32_refine", 1e-12)
    assert info["status"] == 0, info
    f = ctx.eval_poly(c, k, _dev(pb.points[:, 0]), _dev(pb.points[:, 1])).cpu().numpy()
    f_ref = PO.evaluate_poly(c_ref, k_ref, pb.centres, pb.points, pb.R, pb.kernel)
    assert O.rel_err(f, f_ref) <= MIXED_BAR
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("box", [(0.0, 0.0, 1.0), (3.0, -2.0, 0.25)])
def test_poly_reproduces_linear_data(prec, box):
    """h = a_x x + a_y y + a_0 is fitted by the polynomial alone: c = 0, k = a (the least-squares
    solution is unique and exact), also on a box away from the origin. Bar: the FP64 path's
    rounding moves the solution by up to 1e-14 kappa; FP32 + FP64 refinement stops at the
    relative normal residual tol = 1e-13, which bounds the error by tol kappa (kappa of the
    Jacobi-scaled bordered matrix, from the oracle); at least 1e-9, times the coordinates'
    scale."""
    x0, y0, s = box
    rng = np.random.default_rng(5)
    P = rng.random((4000, 2)) * s + (x0, y0)
    C = dg.halton(400) * s + (x0, y0)
    a = np.array([0.7, -1.3, 0.4])
    h = P[:, 0] * a[0] + P[:, 1] * a[1] + a[2]
    R = dg.support_radius(400, 20.0) * s
    tol = 1e-13
    c, k, info, ctx = pkg.fit_poly(P, h, C, R, "w31", prec=prec, tol=tol,
                                   bbox=(x0, y0, x0 + s, y0 + s))
    c, k = c.cpu().numpy(), k.cpu().numpy()
    _, _, d = PO.fit_poly(P, h, C, R, "w31")
    kappa = _kappa(d["K"], d["pinned"])
    scale = max(1.0, abs(x0), abs(y0))
    bar = max(FP64_BAR, (1e-14 if prec == "fp64" else tol) * kappa) * scale
    assert np.abs(c).max() <= bar, (np.abs(c).max(), bar, kappa)
    np.testing.assert_allclose(k, a, rtol=0, atol=bar)
    ctx.close()


def test_poly_pinned_centre_far_from_data():
    pb = dg.config_small(34, 3000, 300)
    C = pb.centres.copy()
    C[7] = (0.5, 0.5)
    keep = np.hypot(pb.points[:, 0] - 0.5, pb.points[:, 1] - 0.5) > 2 * pb.R
    P, h = pb.points[keep], pb.h[keep]
    c_ref, k_ref, d = PO.fit_poly(P, h, C, pb.R, pb.kernel)
    c, k, info, ctx = pkg.fit_poly(P, h, C, pb.R, pb.kernel, prec="fp64", tol=1e-14)
    c, k = c.cpu().numpy(), k.cpu().numpy()
    assert info["pinned"] == int(d["pinned"].sum()) >= 1
    assert c[7] == 0.0
    bar = max(FP64_BAR, 1e-14 * _kappa(d["K"], d["pinned"]))
    ref = np.concatenate([c_ref, k_ref])
    assert np.abs(np.concatenate([c, k]) - ref).max() <= bar * np.abs(ref).max()
    ctx.close()


def test_poly_table4_synthetic(golden_dir):
    """Table 4's synthetic errors with the linear polynomial through the GPU path: 1089 Halton
    points carrying Franke's function, 81 Halton reference points, alpha from Table 3. The
    phi_3,3 case (alpha = 0.25: every support covers the domain several times over) has a
    bordered matrix of condition ~1e18, beyond FP64 normal equations; the oracle's pin solves it
    by QR, and it is left out here."""
    rows = [l.split() for l in open(os.path.join(golden_dir, "table4_synthetic_linear.txt"))
            if l.strip() and not l.startswith("#")]
    P = dg.halton(1089)
    h = dg.franke(P[:, 0], P[:, 1])
    C = dg.halton(81)
    for kind, alpha, mae in rows:
        if kind == "w33":
            continue
        R = 1.0 / float(alpha)
        c, k, info, ctx = pkg.fit_poly(P, h, C, R, kind, prec="fp64", tol=1e-13, min_support=0,
                                       maxit=100000)
        f = ctx.eval_poly(c, k, _dev(P[:, 0]), _dev(P[:, 1])).cpu().numpy()
        got = O.error_measures(f, h)["mae"]
        c_ref, k_ref, _ = PO.fit_poly(P, h, C, R, kind, min_support=0, method="qr")
        ref = O.error_measures(PO.evaluate_poly(c_ref, k_ref, C, P, R, kind), h)["mae"]
        assert abs(got - float(mae)) <= 0.15 * float(mae), (kind, got, mae)
        assert abs(got - ref) <= 1e-6 * ref, (kind, got, ref)
        ctx.close()


def test_poly_argument_errors():
    pb = dg.config_small(35, 2000, 200)
    ctx = pkg.Context()
    ctx.bin(_dev(pb.centres[:, 0]), _dev(pb.centres[:, 1]), _dev(pb.points[:, 0]),
            _dev(pb.points[:, 1]), _dev(pb.h), pb.R)
    ctx.assemble("w31", "fp64")
    with pytest.raises(pkg.RBFError) as e:
        ctx.solve_poly()                      # no polynomial blocks assembled
    assert "RBF_ERR_ARG" in str(e.value)
    ctx.close()
    # collinear points: P^T P is singular, no linear polynomial is determined
    x = np.linspace(0.05, 0.95, 3000)
    P = np.stack([x, 0.5 + 0 * x], 1)
    C = np.stack([np.linspace(0.05, 0.95, 60), 0.5 + np.zeros(60)], 1)
    with pytest.raises(pkg.RBFError) as e:
        pkg.fit_poly(P, np.sin(4 * x), C, 0.05, "w31", prec="fp64")
    assert "RBF_ERR_ARG" in str(e.value)
