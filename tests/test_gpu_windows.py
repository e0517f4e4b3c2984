"""GPU parity of the moving-window fit (rbf_bin_windows + rbf_assemble + rbf_solve_tiles +
rbf_eval_windows(_grid)) against oracle/window_oracle.py on the same seeded inputs.

Bars: window membership exact (each window's centres are the oracle's, integer); the weights
of each window to max(1e-9, 1e-14 kappa_w) relative (kappa_w: condition number of the window's
Jacobi-scaled B) in FP64; the blended surface at the data points and on a grid to 1e-9 (FP64)
and 1e-6 (FP32 + FP64 refinement), or 1e-14 max_w kappa_w where that is larger (a window's
surface is no better determined than its weights; with a margin of 0 on clustered data a
window can be much worse conditioned than the whole domain); one window equals the
single-system fit."""
import numpy as np
import pytest

import datagen as dg
import oracle as O
from oracle import window_oracle as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1806_07884_gb300 as pkg  # noqa: E402

FP64_BAR = 1e-9
MIXED_BAR = 1e-6


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _kappa(P, h, C, R, kind, min_support=3):
    A = O.design_matrix(P, C, R, kind)
    B, _ = O.normal_system(A, h)
    free = ~O.pinned_mask(A, min_support)
    Bd = B.toarray()[free][:, free]
    if Bd.size == 0:
        return 1.0
    d = np.sqrt(np.diag(Bd))
    ev = np.linalg.eigvalsh(Bd / d[:, None] / d[None, :])
    return float(ev[-1] / ev[0])


# name: (problem, wx, wy, overlap / R, margin / R)
CASES = {
    "franke_3x2": (lambda: dg.config_franke(seed=81, N=6000, M=600), 3, 2, 2.0, 1.0),
    "terrain_2x3": (lambda: dg.config_terrain(seed=82, N=20000, M=2000), 2, 3, 3.0, 1.0),
    "terrain_4x3_margin2": (lambda: dg.config_terrain(seed=86, N=20000, M=2000), 4, 3, 1.0, 2.0),
    "uniform_3x3_no_overlap": (lambda: dg.config_small(83, 8000, 600), 3, 3, 0.0, 1.0),
    "franke_2x2_no_margin": (lambda: dg.config_franke(seed=87, N=6000, M=600), 2, 2, 1.0, 0.0),
}


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("case", list(CASES))
def test_windows_match_the_oracle(case, prec):
    make, wx, wy, d_in_R, m_in_R = CASES[case]
    pb = make()
    d, m = d_in_R * pb.R, m_in_R * pb.R
    c, info, tinfo, ctx = pkg.fit_windows(pb.points, pb.h, pb.centres, pb.R, wx, wy, d,
                                          pb.kernel, prec=prec, bbox=pb.bbox, margin=m,
                                          tol=1e-14 if prec == "fp64" else 1e-12)
    assert info["status"] == 0, info
    fits = W.fit_windows(pb.points, pb.h, pb.centres, pb.R, pb.bbox, wx, wy, d, m, pb.kernel)
    wins = W.windows(pb.points, pb.centres, pb.bbox, wx, wy, d, m)
    idx = ctx.window_centres().cpu().numpy()
    cg = c.cpu().numpy()
    assert len(idx) == sum(len(ci) for ci, _ in fits)
    at = 0
    kmax = 1.0
    for w, ((ci, cw), (pi, _)) in enumerate(zip(fits, wins)):
        seg = idx[at:at + len(ci)]
        order = np.argsort(seg)
        np.testing.assert_array_equal(seg[order], ci)          # membership: exact
        if len(pi) > 0:
            kap = _kappa(pb.points[pi], pb.h[pi], pb.centres[ci], pb.R, pb.kernel)
            kmax = max(kmax, kap)
            if prec == "fp64":
                got = cg[at:at + len(ci)][order]
                assert O.rel_err(got, cw) <= max(FP64_BAR, 1e-14 * kap), (w, kap)
        at += len(ci)
    bar = max(FP64_BAR if prec == "fp64" else MIXED_BAR, 1e-14 * kmax)
    f = ctx.eval_windows(c, _dev(pb.points[:, 0]), _dev(pb.points[:, 1])).cpu().numpy()
    f_ref = W.evaluate_windows(fits, pb.centres, pb.points, pb.R, pb.bbox, wx, wy, d, pb.kernel)
    assert O.rel_err(f, f_ref) <= bar, (O.rel_err(f, f_ref), kmax)
    n = 49
    g = ctx.eval_windows_grid(c, n, n, pb.bbox).cpu().numpy()
    g_ref = W.evaluate_windows_grid(fits, pb.centres, pb.R, pb.bbox, wx, wy, d, pb.kernel, n)
    assert O.rel_err(g, g_ref) <= bar, (O.rel_err(g, g_ref), kmax)
    ctx.close()


def test_one_window_is_the_single_system_fit():
    pb = dg.config_franke(seed=84, N=5000, M=500)
    c, info, _, ctx = pkg.fit_windows(pb.points, pb.h, pb.centres, pb.R, 1, 1, 0.1, pb.kernel,
                                      prec="fp64", tol=1e-14)
    idx = ctx.window_centres().cpu().numpy()
    np.testing.assert_array_equal(np.sort(idx), np.arange(pb.M))
    c1, _, ctx1 = pkg.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel, prec="fp64", tol=1e-14)
    cw = np.empty(pb.M)
    cw[idx] = c.cpu().numpy()
    assert O.rel_err(cw, c1.cpu().numpy()) <= FP64_BAR
    g = ctx.eval_windows_grid(c, 33, 33).cpu().numpy()
    g1 = ctx1.eval_grid(c1, 33, 33).cpu().numpy()
    assert O.rel_err(g, g1) <= FP64_BAR
    ctx.close()
    ctx1.close()


def test_many_windows_use_the_per_item_atomic_path():
    """More than 4096 windows: the items are counted and scattered with one global atomic per
    (item, window) instead of the block-aggregated counts; membership and the surface at the
    data points as in the parity cases (FP64)."""
    pb = dg.config_small(88, 200000, 20000)
    wx = wy = 65
    d, m = 0.5 * pb.R, pb.R
    c, info, _, ctx = pkg.fit_windows(pb.points, pb.h, pb.centres, pb.R, wx, wy, d, pb.kernel,
                                      prec="fp64", bbox=pb.bbox, margin=m, tol=1e-13)
    assert info["status"] == 0, info
    wins = W.windows(pb.points, pb.centres, pb.bbox, wx, wy, d, m)
    idx = ctx.window_centres().cpu().numpy()
    at = 0
    for _, ci in wins:
        np.testing.assert_array_equal(np.sort(idx[at:at + len(ci)]), ci)
        at += len(ci)
    assert at == len(idx)
    fits = W.fit_windows(pb.points, pb.h, pb.centres, pb.R, pb.bbox, wx, wy, d, m, pb.kernel)
    Q = pb.points[::10]
    f = ctx.eval_windows(c, _dev(Q[:, 0]), _dev(Q[:, 1])).cpu().numpy()
    f_ref = W.evaluate_windows(fits, pb.centres, Q, pb.R, pb.bbox, wx, wy, d, pb.kernel)
    assert O.rel_err(f, f_ref) <= 1e-8
    ctx.close()


def test_window_errors():
    pb = dg.config_small(85, 2000, 60, K=1.0)
    ctx = pkg.Context()
    args = [_dev(pb.centres[:, 0]), _dev(pb.centres[:, 1]), _dev(pb.points[:, 0]),
            _dev(pb.points[:, 1]), _dev(pb.h), pb.R]
    with pytest.raises(pkg.RBFError) as e:       # many of 100 x 100 windows hold no centre
        ctx.bin_windows(*args, (0.0, 0.0, 1.0, 1.0), 100, 100, 0.0, 0.0)
    assert "RBF_ERR_ARG" in str(e.value)
    for bad in [((0.0, 0.0, 0.0, 1.0), 2, 2, 0.1), ((0.0, 0.0, 1.0, 1.0), 0, 2, 0.1),
                ((0.0, 0.0, 1.0, 1.0), 2, 2, -0.1), ((0.0, 0.0, 1.0, 1.0), 300, 300, 0.1),
                ((0.0, 0.0, 1.0, 1.0), 2, 2, 0.1, -1e-3), ((0.0, 0.0, 1.0, 1.0), 2, 2, 0.1, float("inf"))]:
        with pytest.raises(pkg.RBFError) as e:
            ctx.bin_windows(*args, *bad)
        assert "RBF_ERR_ARG" in str(e.value)
    # a plain binning afterwards leaves the window layout behind
    ctx.bin_windows(*args, (0.0, 0.0, 1.0, 1.0), 2, 2, 2 * pb.R)
    ctx.bin(*args)
    ctx.assemble(pb.kernel, "fp64")
    with pytest.raises(pkg.RBFError):
        ctx.eval_windows_grid(torch.zeros(pb.M, dtype=torch.float64, device="cuda"), 4, 4)
    ctx.close()
