"""Pins of the learned-confidence oracle against things other than itself:
a library's bfloat16 conversion and 2-D correlation, hand-derived features,
finite differences of the loss, closed forms of the first Adam steps and of
networks whose weights route one input value through."""
import os

import numpy as np
import pytest

from oracle import confnet_oracle as co

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "confnet_features.txt")
VISIBILITY = os.path.join(os.path.dirname(__file__), "golden", "visibility_margin.txt")


def test_bf16_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200000) * 5).astype(np.float32)
    # exact ties between two bfloat16 values, both parities of the kept bit
    ties = (np.arange(1, 2000, dtype=np.float32) * np.float32(2 ** -8) + np.float32(1.0))
    x = np.concatenate([x, ties, -ties])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(co.bf16(x), ref)


def test_bf16_hand_values():
    v = co.bf16(np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -9, 255.0, 257.0, 0.0]))
    assert list(v) == [1.0, 1.0, 1 + 2 ** -6, 1.0, 255.0, 256.0, 0.0]


def test_conv_matches_library_correlation():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    a = rng.standard_normal((7, 9, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    got = co._conv3x3(a, w)
    for o in range(4):
        ref = sum(signal.correlate2d(a[:, :, c], w[o, :, :, c], mode="same", boundary="fill")
                  for c in range(3))
        assert np.allclose(got[:, :, o], ref, atol=1e-12)


def _golden_cases():
    cases = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        parts = [p.strip() for p in line.split("|")]
        name, D, x, c = parts[0].split()
        L = [np.array([int(v) for v in p.split()], dtype=np.int64) for p in parts[1:9]]
        exp = [int(v) for v in parts[9].split()]
        cases.append((name, int(D), int(x), int(c), L, exp))
    return cases


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c[0])
def test_features_hand_cases(case):
    _, D, x, c, L, exp = case
    W = x + 1
    vols = [np.zeros((1, W, D), dtype=np.int64) for _ in range(8)]
    for r in range(8):
        vols[r][0, x] = L[r]
    S = sum(vols)
    cost = np.zeros((1, W, D), dtype=np.uint8)
    d_star = exp[4]
    cost[0, x, d_star] = c
    feat, ds = co.features(S, vols, cost)
    assert int(ds[0, x]) == d_star
    scales = [1024, 256, 256, 16, 128, 64, 64, 16]
    assert list(feat[0, x]) == [float(co.bf16(e / s)) for e, s in zip(exp, scales)]


def _visibility_cases():
    cases = []
    for line in open(VISIBILITY):
        if line.startswith("#") or not line.strip():
            continue
        name, row, exp = (p.strip() for p in line.split("|"))
        cases.append((name, [int(v) for v in row.split()], [int(v) for v in exp.split()]))
    return cases


@pytest.mark.parametrize("case", _visibility_cases(), ids=lambda c: c[0])
def test_visibility_margin_hand_rows(case):
    _, row, exp = case
    assert len(row) == len(exp)
    assert list(co.visibility_margin(np.array([row]))[0]) == exp


@pytest.mark.parametrize("case", _visibility_cases(), ids=lambda c: c[0])
def test_visibility_margin_through_features(case):
    """Channel 7 of the features on cost curves whose single minimum sits at
    the row's winners (in L0 only), and rows stacked: each row on its own."""
    _, row, exp = case
    W, D = len(row), max(row) + 2
    vols = [np.zeros((2, W, D), dtype=np.int64) for _ in range(8)]
    for y, shift in ((0, 0), (1, 1)):
        for x, d in enumerate(row):
            dd = min(d + shift, D - 1) if y == 1 else d
            vols[0][y, x] = 50 + 3 * np.abs(np.arange(D) - dd)
    feat, ds = co.features(sum(vols), vols, np.zeros((2, W, D), dtype=np.uint8))
    assert list(ds[0]) == row
    assert list(feat[0, :, 7]) == [float(co.bf16(e / 16)) for e in exp]
    assert np.array_equal(feat[1, :, 7], co.bf16(co.visibility_margin(ds[1:2])[0] / 16))


def test_visibility_margin_step_closed_form():
    """A foreground step of height J at column x0 hides the J background
    pixels left of it: v(x) = (x0 - d_f) - (x - d_b) there, 1 elsewhere."""
    for d_b, d_f, x0, W in ((3, 7, 20, 40), (0, 12, 30, 50), (5, 6, 10, 16)):
        row = np.array([[d_b] * x0 + [d_f] * (W - x0)])
        v = co.visibility_margin(row)[0]
        J = d_f - d_b
        for x in range(W):
            if x == W - 1:
                want = 16
            elif x0 - J <= x < x0:
                want = max((x0 - d_f) - (x - d_b), -16)
            else:
                want = 1
            assert v[x] == want, (d_b, d_f, x0, x)


def test_single_tap_network_routes_one_value():
    """Weights zero except one tap per layer: the logit is feature 0 moved by
    the taps' offsets (zero outside the image), through three ReLUs."""
    H, W = 6, 7
    rng = np.random.default_rng(2)
    feat = co.bf16(rng.uniform(0, 2, size=(H, W, co.F)))
    theta = np.zeros(co.param_count())
    layers = co.split_params(theta)
    (w1, _), (w2, _), (w3, _), (w4, b4) = layers
    w1[0, 1, 1, 0] = 1.0          # centre tap
    w2[0, 0, 1, 0] = 1.0          # tap (ky=0): reads the row above
    w3[0, 1, 2, 0] = 1.0          # tap (kx=2): reads the column to the right
    w4[0, 1, 1, 0] = 1.0
    b4[0] = 0.25
    z, _ = co.forward(theta, feat)
    exp = np.full((H, W), 0.25)
    for y in range(H):
        for x in range(W):
            yy, xx = y - 1, x + 1
            if 0 <= yy < H and 0 <= xx < W:
                exp[y, x] += feat[yy, xx, 0]
    assert np.array_equal(z, exp)


def test_loss_at_zero_logits_is_log2():
    labels = np.array([[[0, 1, 255], [1, 1, 0]]], dtype=np.uint8)
    assert abs(co.loss(np.zeros(labels.shape), labels, 3.0) - np.log(2.0)) < 1e-15


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    B, H, W = 2, 5, 6
    feats = rng.uniform(0, 1.5, size=(B, H, W, co.F))
    labels = rng.integers(0, 2, size=(B, H, W)).astype(np.uint8)
    labels[0, 0, 0] = 255
    theta = np.concatenate([np.concatenate([rng.normal(0, np.sqrt(2 / (9 * ci)), 9 * ci * co_),
                                            rng.normal(0, 0.1, co_)])
                            for ci, co_ in co.LAYERS])
    L, g = co.loss_and_grads(theta, feats, labels, 2.5, round_bf16=False)
    assert abs(L - co.loss(np.stack([co.forward(theta, f, False)[0] for f in feats]), labels,
                           2.5)) < 1e-15
    # a sample of weights and every bias of every layer
    idx, o = [], 0
    for ci, co_ in co.LAYERS:
        nw = 9 * ci * co_
        idx += list(o + rng.choice(nw, size=12, replace=False)) + list(range(o + nw, o + nw + co_))
        o += nw + co_
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = co.loss_and_grads(tp, feats, labels, 2.5, round_bf16=False)
        lm, _ = co.loss_and_grads(tm, feats, labels, 2.5, round_bf16=False)
        num = (lp - lm) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, g[i])


def test_adam_closed_forms():
    rng = np.random.default_rng(4)
    g = rng.standard_normal(50)
    theta = rng.standard_normal(50)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    # first step: bias-corrected moments are g and g^2
    t1, m, v = co.adam(theta, np.zeros(50), np.zeros(50), g, 1, lr, b1, b2, eps)
    assert np.allclose(t1, theta - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    # a constant gradient keeps them there: every step moves by the same amount
    t = t1
    for step in range(2, 6):
        t_next, m, v = co.adam(t, m, v, g, step, lr, b1, b2, eps)
        assert np.allclose(t_next - t, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
        t = t_next


def test_learned_mask_rules():
    prob = np.array([[0.9, 0.9, 0.2, 0.95]])
    dstar = np.array([[0, 2, 0, 3]])
    assert list(co.learned_mask(prob, dstar, 0.5)[0]) == [1, 0, 0, 1]
