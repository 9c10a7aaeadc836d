"""Whole-path pins for the oracle on the tiny fronto-parallel plane scenes
(64x48, D=16, planes at disparities 3, 7, 12, census 9x7, P1=7, P2=86).

* SGM (Sec. 3.1) recovers the exact integer disparity inside every plane,
  away from plane edges, occlusions and the x < D strip, and the left-right
  check keeps those pixels.
* With subpixel refinement off, the combination (Sec. 3.3, Eq. 4-5) of two
  such maps under an integer 2D shift gives the closed form: the point keeps
  its depth Z = fB/d and moves by (uB/d, vB/d, 0)."""
import numpy as np
import pytest

from paper_1801_04720_gb300 import synth

SEEDS = [0, 1, 2, 3]


def interior_mask(q, sid_left, sid_right, disp, margin=1):
    """Pixels whose census window (+margin) lies on one surface in the left view
    and on the same, unoccluded surface in the right view at x - d."""
    H, W = q.shape
    mx, my = 4 + margin, 3 + margin
    out = np.zeros((H, W), dtype=bool)
    for y in range(my, H - my):
        for x in range(max(q.D, mx), W - mx):
            k = sid_left[y, x]
            d = int(disp[y, x])
            if x - d - mx < 0:
                continue
            if (sid_left[y - my:y + my + 1, x - mx:x + mx + 1] != k).any():
                continue
            if (sid_right[y - my:y + my + 1, x - d - mx:x - d + mx + 1] != k).any():
                continue
            out[y, x] = True
    return out


@pytest.mark.parametrize("seed", SEEDS)
def test_exact_integer_disparity_in_plane_interiors(oracle_mod, seed):
    q = synth.fronto_planes(seed=seed)
    r = oracle_mod.disparity(q.left_t, q.right_t, D=q.D)
    inner = interior_mask(q, q.surface_t, q.extra["sid_right_t"], q.gt_disp0)
    assert inner.sum() > 300
    assert np.array_equal(r["dL"][inner], q.gt_disp0[inner].astype(np.int16))
    assert (r["valid"][inner] == 1).all()
    # subpixel refinement stays within half a pixel of the integer winner
    assert (np.abs(r["dL_sub"][inner] - q.gt_disp0[inner]) <= 0.5).all()


@pytest.mark.parametrize("seed", SEEDS)
def test_scene_flow_closed_form_on_shifted_planes(oracle_mod, seed):
    q = synth.fronto_planes(seed=seed)
    cam = q.camera
    res = oracle_mod.scene_flow(q.images(), q.flow, cam.f, cam.B, cam.cx, cam.cy, D=q.D,
                                subpixel=False)
    H, W = q.shape
    in0 = interior_mask(q, q.surface_t, q.extra["sid_right_t"], q.gt_disp0)
    in1 = interior_mask(q, q.extra["sid_left_t1"], q.extra["sid_right_t1"], q.extra["disp_t1"])
    ys, xs = np.mgrid[0:H, 0:W]
    xt = xs + q.flow[..., 0].astype(int)
    yt = ys + q.flow[..., 1].astype(int)
    inside = (xt >= 0) & (xt < W) & (yt >= 0) & (yt < H)
    sel = in0 & inside
    sel[sel] &= in1[yt[sel], xt[sel]]
    assert sel.sum() > 100
    assert (res["valid"][sel] == 1).all()
    d = q.gt_disp0[sel].astype(np.float64)
    u = q.flow[sel, 0].astype(np.float64)
    v = q.flow[sel, 1].astype(np.float64)
    m = res["motion"][sel]
    assert np.allclose(m[:, 0], u * cam.B / d, rtol=0, atol=1e-12)
    assert np.allclose(m[:, 1], v * cam.B / d, rtol=0, atol=1e-12)
    assert np.allclose(m[:, 2], 0.0, rtol=0, atol=1e-12)
    assert np.allclose(res["point"][sel][:, 2], cam.f * cam.B / d, rtol=0, atol=1e-12)
    # flow that leaves the image is always undefined (Eq. 4)
    xp = xs + q.flow[..., 0]
    yp = ys + q.flow[..., 1]
    outside = (xp < 0) | (xp > W - 1) | (yp < 0) | (yp > H - 1)
    assert (res["valid"][outside] == 0).all()
