"""Pins for the oracle's multi-frame extension (the paper's future work,
Sec. 5: more than two frame pairs, with an intermediate validation).

* Two frames reduce exactly to the combination of Sec. 3.3 (Eq. 4, 5): the
  same validity, the first point its point, P_1 - P_0 its motion.
* A scene at one constant disparity moving by a constant integer 2D shift per
  frame: every valid chain has the closed form P_k = P_0 + k (uB/d, vB/d, 0),
  and a chain is valid exactly while x + k u, y + k v stay in the image.
* Intermediate validation: a disparity removed in an intermediate frame
  invalidates exactly the chains that read it (integer flows read one pixel
  per frame), and no other.
* Bilinear flow on a linear field is exact: the chain follows the closed
  form x_{k+1} = x_k + a + b x_k; flows that return every point to its start
  give P_2 = P_0 when the third map equals the first."""
import numpy as np
import pytest

from paper_1801_04720_gb300 import synth


@pytest.mark.parametrize("seed", [0, 3])
def test_two_frames_are_the_combination(oracle_mod, seed):
    q = synth.fronto_planes(seed=seed)
    c = q.camera
    r = oracle_mod.scene_flow(q.images(), q.flow, c.f, c.B, c.cx, c.cy, D=q.D)
    P, v = oracle_mod.chain([r["t0"]["disp"], r["t1"]["disp"]], [q.flow], c.f, c.B, c.cx, c.cy)
    assert np.array_equal(v, r["valid"])
    m = v == 1
    assert m.sum() > 500
    assert np.array_equal(P[0][m], r["point"][m])
    assert np.array_equal((P[1] - P[0])[m], r["motion"][m])
    assert np.isnan(P[:, ~m]).all()


def test_two_frames_with_fractional_flow(oracle_mod):
    rng = np.random.default_rng(1)
    H, W = 30, 40
    D0 = rng.uniform(2, 20, size=(H, W))
    D1 = rng.uniform(2, 20, size=(H, W))
    D0[rng.random((H, W)) < 0.2] = np.nan
    D1[rng.random((H, W)) < 0.2] = np.nan
    flow = rng.normal(0, 4, size=(H, W, 2)).astype(np.float32)
    s4, motion, point, valid = oracle_mod.combine(D0, D1, flow, 100.0, 0.5, 19.5, 14.5)
    P, v = oracle_mod.chain([D0, D1], [flow], 100.0, 0.5, 19.5, 14.5)
    assert np.array_equal(v, valid)
    m = v == 1
    assert np.array_equal((P[1] - P[0])[m], motion[m])


def _const_scene(K, H, W, d, u, v):
    D = [np.full((H, W), d) for _ in range(K)]
    F = [np.full((H, W, 2), (u, v), dtype=np.float32) for _ in range(K - 1)]
    return D, F


@pytest.mark.parametrize("u,v", [(2, 0), (-1, 1), (3, -2)])
def test_constant_velocity_closed_form(oracle_mod, u, v):
    K, H, W, d, f, B = 5, 20, 30, 8.0, 100.0, 0.5
    D, F = _const_scene(K, H, W, d, u, v)
    cx, cy = (W - 1) / 2, (H - 1) / 2
    P, valid = oracle_mod.chain(D, F, f, B, cx, cy)
    ys, xs = np.mgrid[0:H, 0:W]
    inside = np.ones((H, W), dtype=bool)
    for k in range(K):
        inside &= (xs + k * u >= 0) & (xs + k * u <= W - 1) & (ys + k * v >= 0) & (ys + k * v <= H - 1)
    assert np.array_equal(valid == 1, inside)
    step = np.array([u * B / d, v * B / d, 0.0])
    for k in range(K):
        assert np.allclose(P[k][inside] - P[0][inside], k * step, rtol=0, atol=1e-12)
    assert np.allclose(P[0][inside][:, 2], f * B / d, rtol=0, atol=1e-12)


def test_intermediate_frame_validates_the_chain(oracle_mod):
    K, H, W = 4, 15, 25
    D, F = _const_scene(K, H, W, 6.0, 1, 1)
    _, v_all = oracle_mod.chain(D, F, 100.0, 0.5, 12.0, 7.0)
    D[2] = D[2].copy()
    D[2][7, 10] = np.nan              # reached at frame 2 from (8, 5)
    _, v = oracle_mod.chain(D, F, 100.0, 0.5, 12.0, 7.0)
    lost = (v_all == 1) & (v == 0)
    assert lost.sum() == 1 and lost[5, 8]
    assert ((v == 1) <= (v_all == 1)).all()


def test_bilinear_flow_on_a_linear_field(oracle_mod):
    K, H, W = 3, 12, 60
    a, b = 0.5, 0.25
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float32)
    D = [np.full((H, W), 5.0) for _ in range(K)]
    F0 = np.stack([np.full((H, W), 1.5, dtype=np.float32), np.zeros((H, W), np.float32)], -1)
    F1 = np.stack([(a + b * xs).astype(np.float32), np.zeros((H, W), np.float32)], -1)
    P, valid = oracle_mod.chain(D, [F0, F1], 100.0, 0.5, 0.0, 0.0)
    x1 = xs + 1.5
    x2 = x1 + a + b * x1                       # the linear field, interpolated exactly
    inside = (x1 <= W - 1) & (x2 <= W - 1)
    assert np.array_equal(valid == 1, inside)
    assert np.allclose(P[2][inside][:, 0], x2[inside] * 0.5 / 5.0, rtol=0, atol=1e-6)


def test_flows_that_return_give_back_the_start(oracle_mod):
    rng = np.random.default_rng(2)
    K, H, W = 3, 20, 20
    D0 = rng.uniform(3, 9, size=(H, W))
    D = [D0, np.full((H, W), 4.0), D0]
    sh = rng.integers(-2, 3, size=(H, W, 2)).astype(np.float32)
    ys, xs = np.mgrid[0:H, 0:W]
    back = np.zeros_like(sh)
    tx = np.clip(xs + sh[..., 0], 0, W - 1).astype(int)
    ty = np.clip(ys + sh[..., 1], 0, H - 1).astype(int)
    back[ty, tx] = -sh                                   # where each point lands, the way home
    ok_map = np.zeros((H, W), dtype=bool)
    ok_map[ty, tx] = True
    P, valid = oracle_mod.chain(D, [sh, back], 100.0, 0.5, 9.5, 9.5)
    m = valid == 1
    inside = (xs + sh[..., 0] >= 0) & (xs + sh[..., 0] <= W - 1) & (ys + sh[..., 1] >= 0) & (ys + sh[..., 1] <= H - 1)
    home = m & inside
    # chains whose landing pixel's way home is their own come back exactly
    own = np.zeros((H, W), dtype=bool)
    own[home] = (back[ty[home], tx[home]] == -sh[home]).all(axis=1)
    assert own.sum() > 50
    assert np.array_equal(P[2][own], P[0][own])
