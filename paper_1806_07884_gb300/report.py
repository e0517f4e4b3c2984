"""Fit-quality report of Section 6 (Tables 3 and 4) on top of the library: every fit and every
evaluation runs through the C-ABI; this module only summarises the GPU's results on the host.

Table 4 measures the approximation error at the data points (mean absolute error, a "deviation"
that reads as the variance of the error, a mean relative error) and the density of the LSE
matrix B = A^T A (nonzeros over M^2); Table 3 lists the shape parameter alpha (support radius
1/alpha) chosen per Wendland function.

    m = report.fit_measures(points, h, centres, R, "w31")
    sweep = report.alpha_sweep(points, h, centres, "w31", [0.5, 1.0, 2.0])
"""
from __future__ import annotations

import numpy as np

from . import Context


def measures(f, h):
    """Error of the approximant f against the data h (host arrays): mean absolute error,
    variance and standard deviation of the error, and the mean absolute error over the height
    range (the paper prints no denominator for its relative error; this reading takes the
    range of h)."""
    e = np.asarray(f, np.float64) - np.asarray(h, np.float64)
    rng = float(np.max(h) - np.min(h))
    return dict(mae=float(np.mean(np.abs(e))), var=float(np.var(e)), std=float(np.std(e)),
                mre_range=float(np.mean(np.abs(e)) / rng) if rng > 0 else float("nan"))


def density(ctx: Context):
    """(nonzeros of B, nonzeros / M^2) of the context's last assembly, from its stored upper
    triangle: every off-diagonal nonzero stands for two entries of B."""
    row, col, val, _, _ = ctx.export_upper()
    row, col = row.cpu().numpy(), col.cpu().numpy()
    ndiag = int(np.count_nonzero(row == col))
    nnz = 2 * int(row.size) - ndiag
    return nnz, nnz / float(ctx.M) ** 2


def fit_measures(points, h, centres, R: float, kind: str = "w31", prec: str = "fp64",
                 tol: float = 1e-12, min_support: int = 3, poly: bool = False,
                 bbox=(0.0, 0.0, 1.0, 1.0), device: int = 0):
    """Fit through the library (with the linear polynomial of Eq. 6-10 when poly) and report
    the error at the data points and the LSE-matrix density."""
    import torch
    dev = f"cuda:{device}"
    P = np.ascontiguousarray(points, np.float64)
    C = np.ascontiguousarray(centres, np.float64)

    def d(a):
        return torch.as_tensor(np.ascontiguousarray(a, np.float64), device=dev)

    ctx = Context(device)
    ctx.bin(d(C[:, 0]), d(C[:, 1]), d(P[:, 0]), d(P[:, 1]), d(h), R, bbox)
    if poly:
        ctx.assemble_poly(kind, prec)
        c, k, info = ctx.solve_poly(tol=tol, min_support=min_support, raise_on_fail=False)
    else:
        ctx.assemble(kind, prec)
        c, info = ctx.solve(tol=tol, min_support=min_support, raise_on_fail=False)
    qx, qy = d(P[:, 0]), d(P[:, 1])
    f = (ctx.eval_poly(c, k, qx, qy) if poly else ctx.eval(c, qx, qy)).cpu().numpy()
    out = measures(f, h)
    out["nnz"], out["density"] = density(ctx)
    out["iterations"] = info["iterations"]
    out["status"] = info["status"]
    ctx.close()
    return out


def alpha_sweep(points, h, centres, kind: str, alphas, **kw):
    """fit_measures for each shape parameter alpha (support radius 1 / alpha)."""
    kw.setdefault("min_support", 0)
    kw.setdefault("tol", 1e-13)
    return [(float(a), fit_measures(points, h, centres, 1.0 / float(a), kind, **kw))
            for a in alphas]
