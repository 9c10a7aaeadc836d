"""CPU oracle of the learned confidence path (features of the aggregated cost
curve, a 4-layer 3x3 convolutional network, its loss, gradients and the Adam
update).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline legs may import this module; the CUDA product path never
calls it and shares no code with it.

The paper has no learned component: it keeps a disparity where the left-right
check of Sec. 3.1 passes.  This path replaces the right-image SGM pass with a
small network that predicts that check's outcome from the left pass alone,
trained on labels made by the check itself.  Everything here is therefore a
definition of this library's own, written out plainly in float64:

* ``features``: eight per-pixel channels of the aggregated cost curve S of
  the left pass (the eight-path sum of Sec. 3.1), each an integer divided by a
  power of two, rounded to bfloat16 (round to nearest, ties to even).
* ``forward``: z_l = b_l + conv3x3(a_{l-1}, bf16(W_l)) with zero padding,
  a_l = bf16(relu(z_l)) for l = 1..3, logit z_4, probability sigmoid(z_4).
* ``loss_and_grads``: weighted binary cross-entropy on the logits and its
  exact gradients (the bf16 rounding of activations is taken as identity in
  the backward pass).
* ``adam``: Adam with bias correction (Kingma and Ba 2015).

With ``round_bf16=False`` every rounding is skipped, which makes the network
a smooth function of its parameters away from the ReLU kinks; the tests pin
the backward pass against finite differences in that mode.
"""
from __future__ import annotations

import numpy as np

F = 8           # feature channels
C = 32          # hidden channels
LAYERS = [(F, C), (C, C), (C, C), (C, 1)]   # (input channels, output channels)
# Aggregation groups of the eight directions (bit order of the path mask):
# the horizontal pair, the three downward and the three upward paths.
GROUP_H = (0, 1)
GROUP_DOWN = (2, 4, 7)
GROUP_UP = (3, 5, 6)


def param_count() -> int:
    return sum(9 * ci * co + co for ci, co in LAYERS)


def split_params(theta: np.ndarray):
    """Flat parameter vector -> [(W [co][3][3][ci], b [co])] per layer."""
    out, o = [], 0
    for ci, co in LAYERS:
        w = theta[o:o + 9 * ci * co].reshape(co, 3, 3, ci)
        o += 9 * ci * co
        b = theta[o:o + co]
        o += co
        out.append((w, b))
    assert o == theta.size
    return out


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (8 significant bits, ties to even),
    returned as float64.  Written from the definition: with x = m 2^e and
    0.5 <= |m| < 1, keep rint(m 2^8) / 2^8 (numpy's rint rounds halves to
    even).  The values here stay far inside bfloat16's normal range."""
    v = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(v)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def _first_argmin(v: np.ndarray) -> np.ndarray:
    return np.argmin(v, axis=-1)       # numpy returns the first minimum


def features(S: np.ndarray, L: list[np.ndarray], cost: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Features of the left pass.

    S: int [H][W][D], the sum of all eight L_r; L: the eight L_r volumes in
    path-mask order; cost: uint8 [H][W][D].  Returns (feat float64 [H][W][8]
    rounded to bf16, d* int [H][W]).  With d* the first argmin of S and
    S0 = S(d*):
      f0 = S0 / 1024
      f1 = (S2 - S0) / 256, S2 = min of S(d) over |d - d*| >= 2 (S0 if none)
      f2 = curvature / 256: S(d*-1) + S(d*+1) - 2 S0 inside, 2 (S(nb) - S0)
           at an end of the range with its single neighbour nb, 0 if D = 1
      f3 = path disagreement / 16: sum over the three path groups
           (horizontal, downward, upward) of min(|d*_g - d*|, 16), d*_g the
           first argmin of the group's summed L_r
      f4 = d* / 128
      f5 = clamp(x - d*, 0, 64) / 64
      f6 = C(d*) / 64
      f7 = visibility margin / 16 (see visibility_margin): how far the
           pixel's match in the right image lies left of every match of the
           pixels to its right in the same row."""
    S = np.asarray(S, dtype=np.int64)
    H, W, D = S.shape
    ds = _first_argmin(S)
    feat = np.zeros((H, W, F), dtype=np.float64)
    for y in range(H):
        for x in range(W):
            s = S[y, x]
            d = int(ds[y, x])
            s0 = int(s[d])
            far = [int(s[k]) for k in range(D) if abs(k - d) >= 2]
            s2 = min(far) if far else s0
            if D == 1:
                curv = 0
            elif d == 0:
                curv = 2 * (int(s[1]) - s0)
            elif d == D - 1:
                curv = 2 * (int(s[D - 2]) - s0)
            else:
                curv = int(s[d - 1]) + int(s[d + 1]) - 2 * s0
            dis = 0
            for g in (GROUP_H, GROUP_DOWN, GROUP_UP):
                sg = sum(np.asarray(L[r][y, x], dtype=np.int64) for r in g)
                dis += min(abs(int(np.argmin(sg)) - d), 16)
            feat[y, x] = [s0 / 1024, (s2 - s0) / 256, curv / 256, dis / 16, d / 128,
                          min(max(x - d, 0), 64) / 64, int(cost[y, x, d]) / 64, 0.0]
    feat[:, :, 7] = visibility_margin(ds) / 16
    return bf16(feat), ds


def visibility_margin(ds: np.ndarray) -> np.ndarray:
    """Occlusion test on the left winners alone (the uniqueness reading of the
    left-right check of Sec. 3.1).  Pixel x of a row matches right-image
    column u(x) = x - d*(x).  A pixel x' > x whose match lies at or left of
    u(x) hides x from the right camera, so with m(x) = min over x' > x of
    u(x') the margin is v(x) = m(x) - u(x), clamped to [-16, 16]; v <= 0 means
    occluded, v = 1 on a fronto-parallel surface, and the last pixel of a row
    (no x' > x) gets 16.  Returns int [H][W]."""
    ds = np.asarray(ds, dtype=np.int64)
    H, W = ds.shape
    v = np.full((H, W), 16, dtype=np.int64)
    for y in range(H):
        m = None                       # min of u(x') over the pixels right of x
        for x in range(W - 1, -1, -1):
            u = x - int(ds[y, x])
            if m is not None:
                v[y, x] = min(max(m - u, -16), 16)
            m = u if m is None else min(m, u)
    return v


def _conv3x3(a: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Zero-padded 3x3 cross-correlation: out[y,x,co] = sum over (ky, kx, ci)
    of w[co,ky,kx,ci] * a[y+ky-1, x+kx-1, ci].  a: [H][W][ci]."""
    H, W, _ = a.shape
    p = np.zeros((H + 2, W + 2, a.shape[2]))
    p[1:-1, 1:-1] = a
    out = np.zeros((H, W, w.shape[0]))
    for ky in range(3):
        for kx in range(3):
            out += np.tensordot(p[ky:ky + H, kx:kx + W], w[:, ky, kx, :], axes=([2], [1]))
    return out


def forward(theta: np.ndarray, feat: np.ndarray, round_bf16: bool = True):
    """Network forward on one image of features [H][W][F].

    Returns (logit [H][W], activations [a0, a1, a2, a3]); a0 is the input."""
    rnd = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    acts = [rnd(feat)]
    layers = split_params(np.asarray(theta, dtype=np.float64))
    for li, (w, b) in enumerate(layers):
        z = _conv3x3(acts[-1], rnd(w)) + b
        if li < 3:
            acts.append(rnd(np.maximum(z, 0.0)))
        else:
            return z[:, :, 0], acts
    raise AssertionError("unreachable")


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-np.asarray(z, dtype=np.float64)))


def bce_weights(labels: np.ndarray, w_neg: float) -> np.ndarray:
    """Per-pixel loss weight: 1 for label 1, w_neg for label 0, 0 for 255."""
    lab = np.asarray(labels)
    return np.where(lab == 1, 1.0, np.where(lab == 0, float(w_neg), 0.0))


def loss(z: np.ndarray, labels: np.ndarray, w_neg: float) -> float:
    """sum(w * (softplus(z) - y z)) / sum(w) over a batch of logits."""
    z = np.asarray(z, dtype=np.float64)
    y = (np.asarray(labels) == 1).astype(np.float64)
    w = bce_weights(labels, w_neg)
    sp = np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))
    return float((w * (sp - y * z)).sum() / w.sum())


def loss_and_grads(theta: np.ndarray, feats: np.ndarray, labels: np.ndarray, w_neg: float,
                   round_bf16: bool = True):
    """Loss and gradient of the loss over a batch: feats [B][H][W][F],
    labels uint8 [B][H][W].  Returns (loss, grad with theta's layout)."""
    theta = np.asarray(theta, dtype=np.float64)
    rnd = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    layers = split_params(theta)
    wr = [rnd(w) for w, _ in layers]
    zs, all_acts = [], []
    for b in range(feats.shape[0]):
        z, acts = forward(theta, feats[b], round_bf16)
        zs.append(z)
        all_acts.append(acts)
    zs = np.stack(zs)
    L = loss(zs, labels, w_neg)
    wts = bce_weights(labels, w_neg)
    y = (np.asarray(labels) == 1).astype(np.float64)
    dz_out = wts * (sigmoid(zs) - y) / wts.sum()           # dL/dz4, [B][H][W]
    grads = [(np.zeros_like(w), np.zeros(w.shape[0])) for w, _ in layers]
    for b in range(feats.shape[0]):
        acts = all_acts[b]
        dz = dz_out[b][:, :, None]                            # [H][W][1]
        for li in (3, 2, 1, 0):
            a_in = acts[li]
            H, W, ci = a_in.shape
            p = np.zeros((H + 2, W + 2, ci))
            p[1:-1, 1:-1] = a_in
            gw, gb = grads[li]
            for ky in range(3):
                for kx in range(3):
                    gw[:, ky, kx, :] += np.tensordot(dz, p[ky:ky + H, kx:kx + W],
                                                     axes=([0, 1], [0, 1]))
            gb += dz.sum(axis=(0, 1))
            if li == 0:
                break
            # dL/da_in(q) = sum over taps and co of w[co,k,ci] dz(q - k + 1)
            dpad = np.zeros((H + 2, W + 2, dz.shape[2]))
            dpad[1:-1, 1:-1] = dz
            da = np.zeros((H, W, ci))
            for ky in range(3):
                for kx in range(3):
                    da += np.tensordot(dpad[2 - ky:2 - ky + H, 2 - kx:2 - kx + W],
                                       wr[li][:, ky, kx, :], axes=([2], [0]))
            dz = da * (a_in > 0)
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return L, flat


def adam(theta, m, v, g, t: int, lr: float, beta1: float, beta2: float, eps: float):
    """One Adam step (bias-corrected moments); returns (theta', m', v')."""
    m2 = beta1 * m + (1.0 - beta1) * g
    v2 = beta2 * v + (1.0 - beta2) * g * g
    mh = m2 / (1.0 - beta1 ** t)
    vh = v2 / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m2, v2


def learned_mask(prob: np.ndarray, dstar: np.ndarray, threshold: float) -> np.ndarray:
    """Accept a pixel iff x - d* >= 0 and prob >= threshold."""
    H, W = dstar.shape
    xs = np.arange(W)[None, :]
    return ((xs - dstar >= 0) & (prob >= threshold)).astype(np.uint8)
