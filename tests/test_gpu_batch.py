"""GPU parity of the batched path (rbf_bin_tiles + rbf_assemble + rbf_solve_tiles): many
independent tiles of uneven size fitted together must give, tile by tile, the oracle's
least-squares fit of that tile alone.

Bars as for one system: integers (support counts, pinned centres) exact; FP64 c to
max(1e-9, 1e-14 kappa) and f at the data points to 1e-9; FP32 + FP64 refinement: f at the
data points and on a grid to 1e-6 (oracle.rel_err, norm-wise per tile)."""
import numpy as np
import pytest
import scipy.sparse

import datagen as dg
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1806_07884_gb300 as pkg  # noqa: E402

FP64_BAR = 1e-9
MIXED_BAR = 1e-6
OK, ERR_ARG, ERR_NOT_CONVERGED = 0, 1, 4


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _moved(pb, x0, y0, s):
    """The same problem on the box [x0, x0 + s] x [y0, y0 + s] (R scaled by s)."""
    P = pb.points * s + (x0, y0)
    C = pb.centres * s + (x0, y0)
    return dg.Problem(P, pb.h.copy(), C, pb.R * s, pb.kernel, bbox=(x0, y0, x0 + s, y0 + s))


def _tiles_small():
    """Uneven tiles: batched-workload tiles of several sizes, a clustered one, a ragged one
    with few centres per support, and one on a shifted, scaled box."""
    pbs = [dg.tile(1000 + k, N=n) for k, n in enumerate((1500, 4200, 2500, 6000))]
    pbs.append(dg.config_small(3, 3000, 260, K=20.0, clustered=True))
    pbs.append(dg.config_small(4, 777, 61, K=9.0))
    pbs.append(_moved(dg.tile(1010, N=2000), 3.0, -2.0, 0.25))
    return pbs


def _problems(pbs):
    return [(pb.points, pb.h, pb.centres, pb.R, pb.bbox) for pb in pbs]


def _kappa(B, pinned):
    free = ~pinned
    Bf = B.toarray()[free][:, free]
    if Bf.size == 0:
        return 1.0
    d = np.sqrt(np.diag(Bf))
    ev = np.linalg.eigvalsh(Bf / d[:, None] / d[None, :])
    return float(ev[-1] / ev[0])


_REF = {}


def _oracle(pb, key):
    if key not in _REF:
        _REF[key] = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
    return _REF[key]


def test_batched_fp64_matches_oracle_per_tile():
    pbs = _tiles_small()
    cs, info, tinfo, ctx = pkg.fit_tiles(_problems(pbs), prec="fp64", tol=1e-14)
    assert info["status"] == OK and info["promoted"] == 0
    for k, pb in enumerate(pbs):
        c_ref, ref = _oracle(pb, ("small", k))
        c = cs[k].cpu().numpy()
        assert tinfo[k]["status"] == OK
        assert tinfo[k]["pinned"] == int(ref["pinned"].sum())
        assert np.all(c[ref["pinned"]] == 0.0)
        assert O.rel_err(c, c_ref) <= max(FP64_BAR, 1e-14 * _kappa(ref["B"], ref["pinned"])), k
        assert O.rel_err(ref["A"] @ c, ref["A"] @ c_ref) <= FP64_BAR, k
    assert info["pinned"] == sum(t["pinned"] for t in tinfo)
    ctx.close()


def test_batched_fp32_refine_surface_matches_oracle():
    # tol 1e-11: the clustered tile is ill-conditioned enough that a 1e-10 normal residual
    # leaves its surface at ~1.6e-6 (the benchmark's workloads use 1e-11 for the same reason)
    pbs = _tiles_small()
    cs, info, tinfo, ctx = pkg.fit_tiles(_problems(pbs), prec="fp32_refine", tol=1e-11)
    assert info["status"] == OK
    for k, pb in enumerate(pbs):
        c_ref, ref = _oracle(pb, ("small", k))
        c = cs[k].cpu().numpy()
        assert tinfo[k]["status"] == OK and tinfo[k]["rel_residual"] <= 1e-11
        assert O.rel_err(ref["A"] @ c, ref["A"] @ c_ref) <= MIXED_BAR, k
        f = O.evaluate_grid(c, pb.centres, pb.R, pb.kernel, 33, pb.bbox)
        f_ref = O.evaluate_grid(c_ref, pb.centres, pb.R, pb.kernel, 33, pb.bbox)
        assert O.rel_err(f, f_ref) <= MIXED_BAR, k
    ctx.close()


def test_batched_assembly_equals_oracle_blocks():
    """The packed system's B is block diagonal by tile and each block is the tile's own
    A^T A: pattern, support counts exact; values to 1e-12 (FP64) of the tile's max |B|."""
    pbs = _tiles_small()[:5]
    tiles, cx, cy, px, py, hh = pkg.pack_tiles(_problems(pbs))
    ctx = pkg.Context()
    ctx.bin_tiles(tiles, *[_dev(a) for a in (cx, cy, px, py, hh)])
    ctx.assemble("w31", "fp64")
    row, col, val, b, sup = [t.cpu().numpy() for t in ctx.export_upper()]
    owner = np.concatenate([np.full(t["M"], k) for k, t in enumerate(tiles)])
    assert np.all(owner[row] == owner[col])                  # no coupling between tiles
    for k, pb in enumerate(pbs):
        t = tiles[k]
        _, ref = _oracle(pb, ("small", k))
        sel = owner[row] == k
        i, j = row[sel] - t["c0"], col[sel] - t["c0"]
        lo, hi = np.minimum(i, j), np.maximum(i, j)
        got = scipy.sparse.coo_matrix((val[sel], (lo, hi)), shape=(t["M"], t["M"])).toarray()
        Bu = scipy.sparse.triu(ref["B"]).toarray()
        assert np.array_equal(got != 0.0, Bu != 0.0), k
        assert np.abs(got - Bu).max() <= 1e-12 * np.abs(Bu).max(), k
        sl = slice(t["c0"], t["c0"] + t["M"])
        np.testing.assert_array_equal(sup[sl], O.support_counts(ref["A"]))
        assert O.rel_err(b[sl], ref["b"]) <= 1e-12
    ctx.close()


def test_batched_equals_single_system_solves():
    """Each tile follows its own CG: the batched FP64 solve gives every tile the weights and
    (within rounding) the iteration count of solving that tile alone. Both solvers sum with
    atomics, so the counts vary from run to run with the summation order: over six runs of
    each, tile 2 took 440-442 iterations, and one single-system run took 431 (2% below); the
    bound allows 4%. A CG with scalars shared by all tiles would give every tile the count
    of the slowest."""
    pbs = _tiles_small()[:4]
    cs, info, tinfo, ctx = pkg.fit_tiles(_problems(pbs), prec="fp64", tol=1e-12)
    for k, pb in enumerate(pbs):
        c1, i1, ctx1 = pkg.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel, prec="fp64",
                               bbox=pb.bbox, tol=1e-12)
        assert O.rel_err(cs[k].cpu().numpy(), c1.cpu().numpy()) <= 1e-8, k
        assert abs(tinfo[k]["iterations"] - i1["iterations"]) <= 2 + 0.04 * i1["iterations"], k
        ctx1.close()
    its = [t["iterations"] for t in tinfo]
    assert len(set(its)) > 1          # uneven tiles stop at different iterations
    assert info["iterations"] == max(its)
    ctx.close()


def test_batched_tile_order_is_free():
    """Tiles listed in another order than their ranges in the arrays give the same fit."""
    pbs = _tiles_small()[:4]
    tiles, cx, cy, px, py, hh = pkg.pack_tiles(_problems(pbs))
    res = []
    for order in (list(range(4)), [2, 0, 3, 1]):
        ctx = pkg.Context()
        ctx.bin_tiles([tiles[k] for k in order], *[_dev(a) for a in (cx, cy, px, py, hh)])
        ctx.assemble("w31", "fp64")
        c, info, tinfo = ctx.solve_tiles(tol=1e-13)
        res.append(c.cpu().numpy())
        ctx.close()
    assert O.rel_err(res[1], res[0]) <= 1e-10


def test_batched_degenerate_tiles():
    """One centre; no data points at all (every centre pinned, c = 0); data far from some
    centres; a tile of one point and one centre -- next to an ordinary tile."""
    rng = np.random.default_rng(5)
    pbs = [dg.tile(1020, N=3000)]
    one = dg.config_small(21, 40, 1, K=1.0)
    one.centres[:] = (0.5, 0.5)
    one.R = 0.4
    pbs.append(one)
    empty = dg.Problem(np.zeros((0, 2)), np.zeros(0), rng.random((7, 2)), 0.3)
    pbs.append(empty)
    far = dg.config_small(22, 1500, 150)
    keep = np.hypot(far.points[:, 0] - 0.3, far.points[:, 1] - 0.7) > 2 * far.R
    far = dg.Problem(far.points[keep], far.h[keep], far.centres, far.R, far.kernel)
    pbs.append(far)
    single = dg.config_small(8, 1, 1, K=1.0)
    single.centres[:] = single.points[0] + 0.01
    pbs.append(single)
    for prec in ("fp64", "fp32_refine"):
        cs, info, tinfo, ctx = pkg.fit_tiles(_problems(pbs), prec=prec, tol=1e-12,
                                             min_support=1 if prec == "fp64" else 3)
        for k, pb in enumerate(pbs):
            c = cs[k].cpu().numpy()
            assert tinfo[k]["status"] == OK, (prec, k)
            if pb.N == 0:
                assert np.all(c == 0.0) and tinfo[k]["pinned"] == pb.M
                continue
            ms = 1 if prec == "fp64" else 3
            c_ref, ref = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel, min_support=ms)
            assert tinfo[k]["pinned"] == int(ref["pinned"].sum()), (prec, k)
            bar = FP64_BAR if prec == "fp64" else MIXED_BAR
            assert O.rel_err(ref["A"] @ c, ref["A"] @ c_ref) <= bar, (prec, k)
        ctx.close()


def test_batched_argument_errors():
    pbs = _tiles_small()[:2]
    tiles, cx, cy, px, py, hh = pkg.pack_tiles(_problems(pbs))
    d = [_dev(a) for a in (cx, cy, px, py, hh)]
    ctx = pkg.Context()
    bad = [dict(t) for t in tiles]
    bad[1]["c0"] -= 1                               # overlapping centre ranges
    with pytest.raises(pkg.RBFError) as e:
        ctx.bin_tiles(bad, *d)
    assert "RBF_ERR_ARG" in str(e.value)
    bad = [dict(t) for t in tiles]
    bad[1]["p0"] += 1                               # a gap in the point ranges
    bad[1]["N"] -= 1
    with pytest.raises(pkg.RBFError):
        ctx.bin_tiles(bad, *d)
    bad = [dict(t) for t in tiles]
    bad[0]["R"] = 0.0
    with pytest.raises(pkg.RBFError):
        ctx.bin_tiles(bad, *d)
    ctx.bin_tiles(tiles, *d)
    ctx.assemble("w31", "fp64")
    with pytest.raises(pkg.RBFError):               # single-system calls on a batch
        ctx.solve()
    with pytest.raises(pkg.RBFError):
        ctx.eval_grid(torch.zeros(ctx.M, dtype=torch.float64, device="cuda"), 8, 8)
    c, info, tinfo = ctx.solve_tiles(tol=1e-12)
    assert info["status"] == OK
    ctx.close()


def test_batched_maxit_per_tile_status():
    pbs = _tiles_small()[:3]
    tiles, cx, cy, px, py, hh = pkg.pack_tiles(_problems(pbs))
    ctx = pkg.Context()
    ctx.bin_tiles(tiles, *[_dev(a) for a in (cx, cy, px, py, hh)])
    ctx.assemble("w31", "fp64")
    c, info, tinfo = ctx.solve_tiles(tol=1e-14, maxit=5, raise_on_fail=False)
    assert info["status"] == ERR_NOT_CONVERGED
    assert all(t["status"] == ERR_NOT_CONVERGED and t["iterations"] == 5 for t in tinfo)
    ctx.close()


def test_batched_warm_start():
    pbs = _tiles_small()[:3]
    tiles, cx, cy, px, py, hh = pkg.pack_tiles(_problems(pbs))
    ctx = pkg.Context()
    ctx.bin_tiles(tiles, *[_dev(a) for a in (cx, cy, px, py, hh)])
    ctx.assemble("w31", "fp64")
    c1, i1, t1 = ctx.solve_tiles(tol=1e-13)
    c2, i2, t2 = ctx.solve_tiles(tol=1e-13, c0=c1 * (1 + 1e-4))
    for a, b in zip(t1, t2):
        assert b["iterations"] < a["iterations"] and b["status"] == OK
    assert O.rel_err(c2.cpu().numpy(), c1.cpu().numpy()) <= 1e-9
    ctx.close()


def test_batched_start_vector_survives_the_autotuner():
    """The first solve of a fresh context tunes its launch configuration by timing CG
    iterations on the solver's own vectors; a start vector must reach the solve intact. From
    a converged FP64 fit every tile starts below its tolerance and takes no step."""
    pbs = _tiles_small()[:4]
    tiles, cx, cy, px, py, hh = pkg.pack_tiles(_problems(pbs))
    d = [_dev(a) for a in (cx, cy, px, py, hh)]
    ctx = pkg.Context()
    ctx.bin_tiles(tiles, *d)
    ctx.assemble("w31", "fp64")
    c1, i1, t1 = ctx.solve_tiles(tol=1e-13)
    ctx.close()
    ctx = pkg.Context()                             # untuned: the autotuner runs first
    ctx.bin_tiles(tiles, *d)
    ctx.assemble("w31", "fp64")
    c2, i2, t2 = ctx.solve_tiles(tol=1e-12, c0=c1)
    assert all(t["iterations"] <= 2 and t["status"] == OK for t in t2), t2
    assert O.rel_err(c2.cpu().numpy(), c1.cpu().numpy()) <= 1e-12
    ctx.close()


def test_batched_promotion_finishes_only_the_unconverged_tiles():
    """FP32 refinement cut short (3 steps to 1e-8): the tiles that converged keep their refined
    iterates, the clustered tile is finished by FP64 CG started from its refined iterate.
    Every tile's returned weights meet the tolerance in the oracle's FP64 normal residual
    (over unpinned centres). FP32 rounding order varies from run to run, so up to four fresh
    contexts are tried for a batch with both kinds of tile."""
    pbs = _tiles_small()
    tiles, cx, cy, px, py, hh = pkg.pack_tiles(_problems(pbs))
    d = [_dev(a) for a in (cx, cy, px, py, hh)]
    tol = 1e-8
    mixed = False
    for attempt in range(4):
        ctx = pkg.Context()
        ctx.bin_tiles(tiles, *d)
        ctx.assemble("w31", "fp32_refine")
        ctx.set_param("max_refinements", 3)
        c, info, tinfo = ctx.solve_tiles(tol=tol)
        ctx.close()
        for k, pb in enumerate(pbs):
            t = tiles[k]
            _, ref = _oracle(pb, ("small", k))
            ck = c[t["c0"]:t["c0"] + t["M"]].cpu().numpy()
            A, free = ref["A"], ~ref["pinned"]
            r = A.T @ (pb.h - A @ ck)
            rel = np.linalg.norm(r[free]) / np.linalg.norm(ref["b"][free])
            assert tinfo[k]["status"] == OK and rel <= 1.5 * tol, (k, rel, tinfo[k])
        pro = [t["promoted"] for t in tinfo]
        assert info["promoted"] == int(any(pro))
        if any(pro) and not all(pro):
            mixed = True
            break
    assert mixed, pro


def test_batched_more_tiles_than_one_worklist_round():
    """1,100 small tiles (more than the 1,024 the work-list build scans per round), FP32 +
    refinement: every tile converges, and sampled tiles match the oracle's fit of that tile
    alone. Tiles stop at different iterations, so the lists are rebuilt many times."""
    rng = np.random.default_rng(11)
    pbs = [dg.tile(70000 + k, N=int(rng.integers(300, 900))) for k in range(1100)]
    cs, info, tinfo, ctx = pkg.fit_tiles(_problems(pbs), prec="fp32_refine", tol=1e-11)
    assert info["status"] == OK
    assert all(t["status"] == OK and t["rel_residual"] <= 1e-11 for t in tinfo)
    its = [t["iterations"] for t in tinfo]
    assert len(set(its)) > 10
    for k in [0, 1, 511, 1023, 1024, 1025, 1099] + list(rng.choice(1100, 5, replace=False)):
        pb = pbs[k]
        c_ref, ref = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
        c = cs[k].cpu().numpy()
        assert O.rel_err(ref["A"] @ c, ref["A"] @ c_ref) <= MIXED_BAR, k
    ctx.close()


def test_autotuner_choice_and_forced_configs_agree():
    pbs = [dg.tile(1030 + k, N=n) for k, n in enumerate((3000, 9000, 5000, 12000))]
    tiles, cx, cy, px, py, hh = pkg.pack_tiles(_problems(pbs))
    ctx = pkg.Context()
    ctx.bin_tiles(tiles, *[_dev(a) for a in (cx, cy, px, py, hh)])
    ctx.assemble("w31", "fp32_refine")
    tu = ctx.autotune()
    assert 1 <= tu["spmv_blocks_per_sm"] <= 8
    assert tu["spmv_chunk"] in (1, 2, 4, 8, 16)
    assert tu["update_threads"] in (128, 256, 512)
    assert tu["us_per_iteration"] > 0.0
    c_auto, info, _ = ctx.solve_tiles(tol=1e-10)
    assert ctx.tuning() == tu                       # the cached choice was used
    refs = [_oracle(pb, ("tune", k)) for k, pb in enumerate(pbs)]
    # chunk 40: SpMV items of more than 32 cells (their cell indices take two loads per lane)
    for bps, chunk, nt in ((1, 1, 128), (2, 8, 512), (3, 16, 256), (2, 40, 256)):
        ctx.set_param("spmv_blocks_per_sm", bps)
        ctx.set_param("spmv_chunk", chunk)
        ctx.set_param("update_threads", nt)
        c, info, tinfo = ctx.solve_tiles(tol=1e-10)
        assert info["status"] == OK
        for k, pb in enumerate(pbs):
            t = tiles[k]
            ck = c[t["c0"]:t["c0"] + t["M"]].cpu().numpy()
            A, c_ref = refs[k][1]["A"], refs[k][0]
            assert O.rel_err(A @ ck, A @ c_ref) <= MIXED_BAR
    with pytest.raises(pkg.RBFError):
        ctx.set_param("update_threads", 384)
    ctx.close()


def test_batched_workload_512_tiles_full_size():
    """The batched workload at its full size (512 tiles, N log-uniform in [2e3, 2e5],
    M = N / 10, phi_3,1, FP32 + FP64 refinement) in the launch configuration the benchmark
    uses: every tile converges to its own tolerance; the smallest tiles match the oracle's
    fit; for sampled centres of the largest tiles the oracle's entry-by-entry FP64 normal
    residual agrees with the convergence the solver reports."""
    pbs = dg.tile_batch(1000, 512)
    cs, info, tinfo, ctx = pkg.fit_tiles(_problems(pbs), prec="fp32_refine", tol=1e-11)
    assert info["status"] == OK
    assert all(t["status"] == OK and t["rel_residual"] <= 1e-11 for t in tinfo)
    order = np.argsort([pb.N for pb in pbs])
    for k in order[:3]:
        pb = pbs[k]
        c_ref, ref = O.fit(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
        c = cs[k].cpu().numpy()
        assert O.rel_err(ref["A"] @ c, ref["A"] @ c_ref) <= MIXED_BAR, k
    rng = np.random.default_rng(0)
    for k in order[-2:]:
        pb = pbs[k]
        so = O.SampledOracle(pb.points, pb.h, pb.centres, pb.R, pb.kernel)
        c = cs[k].cpu().numpy()
        bmax = max(abs(so.b_entry(j)) for j in rng.choice(pb.M, 50, replace=False))
        for j in rng.choice(pb.M, 30, replace=False):
            if so.support(j) >= 3:
                assert abs(so.normal_residual(c, j)) <= 1e-8 * bmax
    ctx.close()


def test_batched_eval_matches_oracle():
    """Batched step (e): each tile's surface on its own grid (inclusive ends) and at its data
    points, from the FP64 batched fit, against the oracle's surface of that tile."""
    pbs = _tiles_small()
    cs, info, tinfo, ctx = pkg.fit_tiles(_problems(pbs), prec="fp64", tol=1e-14)
    c_all = torch.cat(cs)
    fg = ctx.eval_tiles_grid(c_all, 33, 29).cpu().numpy()
    qx = np.concatenate([pb.points[:, 0] for pb in pbs])
    qy = np.concatenate([pb.points[:, 1] for pb in pbs])
    qoff = np.concatenate([[0], np.cumsum([pb.N for pb in pbs])])
    fp = ctx.eval_tiles(c_all, _dev(qx), _dev(qy), qoff).cpu().numpy()
    for k, pb in enumerate(pbs):
        c_ref, ref = _oracle(pb, ("small", k))
        x0, y0, x1, y1 = pb.bbox
        X, Y = np.meshgrid(np.linspace(x0, x1, 33), np.linspace(y0, y1, 29))
        f_ref = O.evaluate(c_ref, pb.centres, np.column_stack([X.ravel(), Y.ravel()]), pb.R,
                           pb.kernel)
        assert O.rel_err(fg[k].ravel(), f_ref) <= FP64_BAR, k
        assert O.rel_err(fp[qoff[k]:qoff[k + 1]], ref["A"] @ c_ref) <= FP64_BAR, k
    with pytest.raises(pkg.RBFError):
        ctx.eval_tiles(c_all, _dev(qx), _dev(qy), qoff[::-1].copy())
    ctx.close()
