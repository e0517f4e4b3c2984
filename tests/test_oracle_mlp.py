"""Pins of the warm-start oracle (oracle/mlp_oracle.py) against values fixed by hand, by
the definitions of BF16 and Adam, and by finite differences -- nothing here retypes the
oracle's formulas."""
import numpy as np
import pytest

import datagen as dg
import oracle as O
from oracle import mlp_oracle as MO


def test_sizes():
    assert MO.NPARAM == 6337 == dg.MLP_NPARAM
    p = dg.mlp_init(0)
    assert p.dtype == np.float32 and p.size == MO.NPARAM
    W1, b1, W2, b2, W3, b3 = MO.unpack(p)
    assert W1.shape == (64, 32) and W2.shape == (64, 64) and W3.shape == (64,)
    assert not b1.any() and not b2.any() and not b3.any()


def test_bf16_round_known_values():
    one = 1.0
    cases = {
        1.0: 1.0,
        -2.5: -2.5,
        one + 2.0 ** -8: 1.0,                       # halfway, kept part even: down
        one + 3 * 2.0 ** -8: one + 2.0 ** -6,       # halfway, kept part odd: up
        one + 2.0 ** -8 + 2.0 ** -20: one + 2.0 ** -7,   # above halfway: up
        one + 2.0 ** -9: 1.0,                       # below halfway: down
        3.140625: 3.140625,                         # representable in BF16
        0.0: 0.0,
    }
    a = np.array(list(cases), np.float32)
    np.testing.assert_array_equal(MO.bf16_round(a), np.array(list(cases.values()), np.float32))
    # the result has at most 8 significant bits
    r = MO.bf16_round(np.random.default_rng(0).normal(size=1000).astype(np.float32))
    assert not (r.view(np.uint32) & 0xFFFF).any()


def test_radial_features_by_hand():
    C = np.array([[0.5, 0.5]])
    R = 0.4
    # distances 0, 0.05 (r = 0.125: bin 2, on the edge), 0.12 (r = 0.3: bin 4),
    # 0.399 (r = 0.9975: bin 15), 0.4 (r = 1: outside), 1.0 (outside)
    d = np.array([0.0, 0.05, 0.12, 0.399, 0.4, 1.0])
    P = np.column_stack([0.5 + d, np.full(d.size, 0.5)])
    h = np.array([1.0, 2.0, 3.0, 5.0, 100.0, 100.0])
    f = MO.radial_features(P, h, C, R, scale=2.0)[0]
    counts = np.zeros(16)
    counts[[0, 2, 4, 15]] = 1
    np.testing.assert_allclose(f[:16], counts / 4)
    means = np.zeros(16)
    means[[0, 2, 4, 15]] = np.array([1.0, 2.0, 3.0, 5.0]) / 2.0
    np.testing.assert_allclose(f[16:], means)
    assert MO.height_scale([3.0, -4.0]) == pytest.approx(np.sqrt(12.5))


def test_radial_features_invariants():
    pb = dg.config_small(31, 3000, 300)
    f = MO.radial_features(pb.points, pb.h, pb.centres, pb.R)
    A = O.design_matrix(pb.points, pb.centres, pb.R)
    n = O.support_counts(A)
    frac = f[:, :16].sum(axis=1)
    np.testing.assert_allclose(frac[n > 0], 1.0, atol=1e-12)
    assert np.all(frac[n == 0] == 0.0)
    # constant heights: every occupied bin's mean height is h / sigma = 1
    fc = MO.radial_features(pb.points, np.full(pb.N, -0.7), pb.centres, pb.R)
    occ = fc[:, :16] > 0
    np.testing.assert_allclose(fc[:, 16:][occ], -1.0, atol=1e-12)
    assert np.all(fc[:, 16:][~occ] == 0.0)


def test_forward_closed_form():
    # W1 selects the first 3 features, W2 the identity, W3 weights 1, 2, 3: with
    # representable (BF16-exact) weights y = b3 + sum_k w_k relu(relu(x_k + b1_k) + b2_k)
    p = np.zeros(MO.NPARAM, np.float32)
    W1, b1, W2, b2, W3, b3 = MO.unpack(p)
    for k in range(3):
        W1[k, k] = 1.0
        W2[k, k] = 1.0
        W3[k] = k + 1.0
    b1[:3] = [0.5, -1.0, 0.0]
    b2[:3] = [0.0, 0.25, -0.5]
    b3[0] = 0.125
    X = np.array([[1.0, 2.0, 3.0] + [9.0] * 29, [-1.0, 0.5, 0.25] + [0.0] * 29])
    want = [0.125 + 1 * 1.5 + 2 * 1.25 + 3 * 2.5, 0.125 + 0 + 2 * 0.25 + 0]
    np.testing.assert_allclose(MO.mlp_forward(p, X), want, rtol=0, atol=1e-15)


def test_gradient_against_finite_differences():
    rng = np.random.default_rng(1)
    p = dg.mlp_init(3).astype(np.float64)
    p[MO.HID * MO.NFEAT: MO.HID * MO.NFEAT + MO.HID] = rng.normal(0, 0.1, MO.HID)   # b1 != 0
    X = rng.normal(size=(40, 32))
    t = rng.normal(size=40)
    L, g = MO.mlp_loss_grad(p, X, t, round_weights=False)
    idx = rng.choice(MO.NPARAM, 200, replace=False)
    eps = 1e-6
    for k in idx:
        e = np.zeros(MO.NPARAM)
        e[k] = eps
        fd = (MO.mlp_loss_grad(p + e, X, t, False)[0] - MO.mlp_loss_grad(p - e, X, t, False)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])
    assert L == pytest.approx(np.mean((MO.mlp_forward(p, X, False) - t) ** 2))


def test_rounded_gradient_is_the_gradient_at_the_rounded_weights():
    rng = np.random.default_rng(2)
    p = dg.mlp_init(4)
    X = rng.normal(size=(30, 32))
    t = rng.normal(size=30)
    pr = p.copy()
    W1, _, W2, _, W3, _ = MO.unpack(pr)
    for w in (W1, W2, W3):
        w[...] = MO.bf16_round(w)
    L1, g1 = MO.mlp_loss_grad(p, X, t, round_weights=True)
    L2, g2 = MO.mlp_loss_grad(pr, X, t, round_weights=False)
    assert L1 == L2
    np.testing.assert_array_equal(g1, g2)


def test_adam_first_steps_by_hand():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    p1, m1, v1 = MO.adam_step(p, np.zeros(3), np.zeros(3), g, 1, 0.01)
    # step 1: bias-corrected m = g, v = g^2, so the step is lr * g / (|g| + eps)
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-15)
    g2 = np.array([0.1, 1.0, 2.0])
    p2, m2, v2 = MO.adam_step(p1, m1, v1, g2, 2, 0.01)
    m = 0.9 * 0.1 * g + 0.1 * g2
    v = 0.999 * 0.001 * g * g + 0.001 * g2 * g2
    np.testing.assert_allclose(m2, m, rtol=1e-15)
    np.testing.assert_allclose(v2, v, rtol=1e-15)
    mh, vh = m / (1 - 0.81), v / (1 - 0.999 ** 2)
    np.testing.assert_allclose(p2, p1 - 0.01 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-14)


def test_oracle_training_reduces_loss():
    """Adam on the oracle's gradient fits a smooth target of the features."""
    rng = np.random.default_rng(5)
    X = rng.normal(size=(256, 32))
    t = np.tanh(X[:, 0]) + 0.5 * X[:, 16]
    p = dg.mlp_init(6).astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0 = MO.mlp_loss_grad(p, X, t)[0]
    for step in range(1, 201):
        L, g = MO.mlp_loss_grad(p, X, t)
        p, m, v = MO.adam_step(p, m, v, g, step, 3e-3)
    assert MO.mlp_loss_grad(p, X, t)[0] < 0.1 * L0
