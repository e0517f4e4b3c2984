"""GPU parity of the learned warm start (rbf_features, rbf_mlp_forward, rbf_mlp_train_step,
rbf_warm_start) against the oracle (oracle/mlp_oracle.py), and the gain it brings.

Bars: per-bin point counts exact (the bin is decided in FP64 on both sides); FP32 features
and network outputs to FP32 accumulation error (1e-5 norm-wise); gradients to 1e-4
norm-wise (FP32 sums over 64 samples per block); one Adam step to the oracle's update."""
import numpy as np
import pytest

import datagen as dg
import oracle as O
from oracle import mlp_oracle as MO

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1806_07884_gb300 as pkg  # noqa: E402
from paper_1806_07884_gb300 import warmstart as W  # noqa: E402


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _binned(pb):
    ctx = pkg.Context()
    C, P = pb.centres, pb.points
    ctx.bin(_dev(C[:, 0]), _dev(C[:, 1]), _dev(P[:, 0]), _dev(P[:, 1]), _dev(pb.h), pb.R, pb.bbox)
    return ctx


def _check_features(feat, ref, n_support):
    counts = np.rint(feat[:, :16] * np.maximum(n_support, 1)[:, None])
    ref_counts = np.rint(ref[:, :16] * np.maximum(n_support, 1)[:, None])
    np.testing.assert_array_equal(counts, ref_counts)              # integers: exact
    assert np.abs(feat - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("case", ["franke", "clustered", "ragged", "terrain"])
def test_features_match_oracle(case):
    pb = {"franke": lambda: dg.config_franke(seed=1, N=5000, M=500),
          "clustered": lambda: dg.config_small(3, 6000, 400, clustered=True),
          "ragged": lambda: dg.config_small(4, 777, 61, K=9.0),
          "terrain": lambda: dg.config_terrain(seed=2, N=20000, M=2000)}[case]()
    ctx = _binned(pb)
    feat, sig = ctx.features()
    ref = MO.radial_features(pb.points, pb.h, pb.centres, pb.R)
    n = O.support_counts(O.design_matrix(pb.points, pb.centres, pb.R))
    _check_features(feat.cpu().numpy().astype(np.float64), ref, n)
    assert abs(float(sig[0]) - MO.height_scale(pb.h)) <= 1e-12 * MO.height_scale(pb.h)
    ctx.close()


def test_features_of_a_batch_per_tile():
    pbs = [dg.tile(2000 + k, N=n) for k, n in enumerate((2500, 6000, 4000))]
    tiles, cx, cy, px, py, hh = pkg.pack_tiles([(p.points, p.h, p.centres, p.R, p.bbox) for p in pbs])
    ctx = pkg.Context()
    ctx.bin_tiles(tiles, *[_dev(a) for a in (cx, cy, px, py, hh)])
    feat, sig = ctx.features()
    feat = feat.cpu().numpy().astype(np.float64)
    for k, pb in enumerate(pbs):
        t = tiles[k]
        ref = MO.radial_features(pb.points, pb.h, pb.centres, pb.R)
        n = O.support_counts(O.design_matrix(pb.points, pb.centres, pb.R))
        _check_features(feat[t["c0"]:t["c0"] + t["M"]], ref, n)
        assert abs(float(sig[k]) - MO.height_scale(pb.h)) <= 1e-12 * MO.height_scale(pb.h)
    ctx.close()


def _random_params(seed):
    rng = np.random.default_rng(seed)
    p = dg.mlp_init(seed).copy()
    W1, b1, W2, b2, W3, b3 = MO.unpack(p)
    b1[:] = rng.normal(0, 0.2, 64)
    b2[:] = rng.normal(0, 0.2, 64)
    b3[:] = 0.3
    return p


def test_forward_matches_oracle():
    rng = np.random.default_rng(3)
    p = _random_params(7)
    X = rng.normal(size=(5000, 32)).astype(np.float32)
    ctx = pkg.Context()
    y = ctx.mlp_forward(_dev(p, torch.float32), _dev(X, torch.float32)).cpu().numpy()
    ref = MO.mlp_forward(p, X.astype(np.float64))
    assert O.rel_err(y, ref) <= 1e-5
    # the BF16 rounding is applied: without it the outputs differ by far more than FP32 error
    assert O.rel_err(MO.mlp_forward(p, X.astype(np.float64), round_weights=False), ref) > 1e-4
    ctx.close()


def test_gradient_and_adam_step_match_oracle():
    rng = np.random.default_rng(4)
    p = _random_params(8)
    X = rng.normal(size=(1000, 32)).astype(np.float32)
    t = rng.normal(size=1000).astype(np.float32)
    ctx = pkg.Context()
    dp, dX, dt = _dev(p, torch.float32), _dev(X, torch.float32), _dev(t, torch.float32)
    grad = torch.empty(MO.NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    ctx.mlp_train_step(dp, None, None, 0, 0.0, dX, dt, grad=grad, loss=loss)
    L, g = MO.mlp_loss_grad(p, X.astype(np.float64), t.astype(np.float64))
    assert abs(float(loss) - L) <= 1e-5 * L
    gg = grad.cpu().numpy()
    assert O.rel_err(gg, g) <= 1e-4
    # a permuted index set gives the same gradient (sample order does not matter)
    idx = _dev(rng.permutation(1000).astype(np.int32), torch.int32)
    grad2 = torch.empty_like(grad)
    ctx.mlp_train_step(dp, None, None, 0, 0.0, dX, dt, idx=idx, grad=grad2)
    assert O.rel_err(grad2.cpu().numpy(), g) <= 1e-4
    # one Adam step
    m = torch.zeros_like(grad)
    v = torch.zeros_like(grad)
    ctx.mlp_train_step(dp, m, v, 1, 1e-3, dX, dt)
    p1, m1, v1 = MO.adam_step(p.astype(np.float64), 0, 0, g, 1, 1e-3)
    big = np.abs(g) > 1e-3 * np.abs(g).max()         # sign-stable entries
    np.testing.assert_allclose(dp.cpu().numpy()[big], p1[big], rtol=0, atol=1e-6)
    np.testing.assert_allclose(m.cpu().numpy(), m1, rtol=1e-4, atol=1e-7 * np.abs(m1).max())
    ctx.close()


def _tiles(seeds, N):
    return [dg.tile(s, N=N) for s in seeds]


def _problems(pbs):
    return [(p.points, p.h, p.centres, p.R, p.bbox) for p in pbs]


# The learned start's measured iteration ratio on the held-out tiles below (FP32 + FP64
# refinement to 1e-10): about 1 -- what the start vector gains is its residual and surface
# error, not CG iterations (tests/test_warmstart_bound.py: a start must be within ~3% of the
# answer in every mode to save 15%).
RATIO_BAND = (0.93, 1.03)


def test_training_reduces_loss_and_what_the_warm_start_gains():
    """Train on 48 solved tiles with the library's own kernels, then start the solver of 8
    held-out tiles from the network's prediction. What it gains: the start vector's normal
    residual and surface error are well below those of c = 0. What it does not: the CG
    iteration count stays about the same -- the network predicts the smooth part of the
    weights, which lies in the large-eigenvalue modes of B that CG resolves in few
    iterations; the oscillating part, in the small-eigenvalue modes that set the iteration
    count, is not a function of the radial statistics. The solve reaches the same fit."""
    train_pbs = _tiles(range(50000, 50048), 12000)
    feat, target, ctx = W.training_set(_problems(train_pbs))
    params, losses = W.train(ctx, feat, target, epochs=12, batch=2048, lr=3e-3, seed=1)
    # losses[0] is the untrained network's; the least-squares weights oscillate from centre
    # to centre, so only part of their variance is a function of the local statistics
    assert losses[-1] < 0.8 * losses[0]
    assert losses[-1] < 0.9 * float(target.double().var())
    ctx.close()
    test_pbs = _tiles(range(60000, 60008), 12000)
    tiles, cx, cy, px, py, hh = pkg.pack_tiles(_problems(test_pbs))
    ctx = pkg.Context()
    ctx.bin_tiles(tiles, *[_dev(a) for a in (cx, cy, px, py, hh)])
    ctx.assemble("w31", "fp32_refine")
    c_cold, i_cold, t_cold = ctx.solve_tiles(tol=1e-10)
    c0 = ctx.warm_start(params)
    # residual of the start vector, per tile, from the oracle
    r0s, e0s = [], []
    for k, pb in enumerate(test_pbs):
        t = tiles[k]
        A = O.design_matrix(pb.points, pb.centres, pb.R)
        cw = c0[t["c0"]:t["c0"] + t["M"]].cpu().numpy()
        r0s.append(np.linalg.norm(A.T @ (pb.h - A @ cw)) / np.linalg.norm(A.T @ pb.h))
        e0s.append(np.linalg.norm(pb.h - A @ cw) / np.linalg.norm(pb.h))
    assert np.median(r0s) < 0.5, r0s          # c = 0 has 1 for both
    assert np.median(e0s) < 0.5, e0s
    c_warm, i_warm, t_warm = ctx.solve_tiles(tol=1e-10, c0=c0)
    it_cold = sum(t["iterations"] for t in t_cold)
    it_warm = sum(t["iterations"] for t in t_warm)
    ratio = it_warm / it_cold
    print(f"learned start / cold start CG iterations on 8 held-out tiles: {it_warm} / {it_cold}"
          f" = {ratio:.4f}")
    assert RATIO_BAND[0] <= ratio <= RATIO_BAND[1], (it_warm, it_cold)
    assert all(t["status"] == 0 for t in t_warm)
    for k, pb in enumerate(test_pbs):
        t = tiles[k]
        A = O.design_matrix(pb.points, pb.centres, pb.R)
        sl = slice(t["c0"], t["c0"] + t["M"])
        assert O.rel_err(A @ c_warm[sl].cpu().numpy(), A @ c_cold[sl].cpu().numpy()) <= 1e-6
    ctx.close()
