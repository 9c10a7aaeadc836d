"""The automotive recipe's ground truth, which the accuracy figures compare
against, agrees with its own renderings: the disparity at t is f B / Z of
the surface the left view sees, and a point carried by the true flow lands
where the t+1 left view shows the same surface at the ground-truth
disparity at t+1 (wherever that surface is still visible there)."""
import numpy as np

import paper_1801_04720_gb300.synth as synth


def _render_with_depths(monkeypatch, **kw):
    casts = []
    orig = synth._cast

    def spy(surfs, W, H, cam, ox):
        out = orig(surfs, W, H, cam, ox)
        casts.append((ox, out[0], out[1]))
        return out

    monkeypatch.setattr(synth, "_cast", spy)
    q = synth.automotive(**kw)
    # views are cast in the order left_t, right_t, left_t1, right_t1
    return q, casts


def test_disparity_at_t_is_the_rendered_depth(monkeypatch):
    q, casts = _render_with_depths(monkeypatch, seed=5, W=320, H=160, D=128, n_segments=6)
    fB = q.camera.f * q.camera.B
    k_t, z_t = casts[0][1], casts[0][2]
    assert np.array_equal(k_t, q.surface_t)
    assert np.allclose(q.gt_disp0, fB / z_t, rtol=1e-6)


def test_flow_and_disparity_at_t1_match_the_t1_rendering(monkeypatch):
    q, casts = _render_with_depths(monkeypatch, seed=6, W=320, H=160, D=128, n_segments=6)
    fB = q.camera.f * q.camera.B
    k_t1, z_t1 = casts[2][1], casts[2][2]
    H, W = q.shape
    ys, xs = np.mgrid[0:H, 0:W]
    x1 = np.rint(xs + q.gt_flow[..., 0]).astype(int)
    y1 = np.rint(ys + q.gt_flow[..., 1]).astype(int)
    inb = (x1 >= 0) & (x1 < W) & (y1 >= 0) & (y1 < H)
    same = np.zeros((H, W), bool)
    same[inb] = k_t1[y1[inb], x1[inb]] == q.surface_t[inb]
    assert same.mean() > 0.3
    d1 = fB / z_t1[y1[same], x1[same]]
    err = np.abs(d1 - q.gt_disp1[same])
    # the nearest pixel centre differs from the exact landing point by up to
    # half a pixel, which a slanted surface turns into a small disparity change
    assert np.median(err) < 0.05
    assert np.percentile(err, 95) < 0.5
    # static background: no motion, flow zero, disparity unchanged
    static = (q.surface_t <= 1)
    assert np.allclose(q.gt_flow[static], 0.0, atol=1e-3)
    assert np.allclose(q.gt_disp1[static], q.gt_disp0[static], rtol=1e-6)
