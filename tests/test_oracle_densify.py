"""Pins for the oracle's densification (the paper's future work, Sec. 5;
Table 1's dense rows come from the benchmark's own fill of a sparse result).

* Hand-worked fills of small grids in both modes (tests/golden/fill.txt).
* Exactness on piecewise-constant rows: every gap inside a constant segment
  takes that constant.
* With a constant guide every edge-aware choice is a tie, which reduces mode
  1 to the background fill; a fully kept map is returned unchanged, and the
  fill is idempotent.
* The background fill equals the evaluation module's own implementation
  (torch, cumulative maxima), written independently of the oracle.
* Dense scene flow: where the sparse result is defined nothing changes; a
  scene at one constant disparity moved by a pure 2D shift gives the closed
  form motion (uB/d, vB/d, 0) at every pixel."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fill.txt")


def _cases():
    cases, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tok = line.split()
        if tok[0] == "case":
            cur = {"name": tok[1], "mode": int(tok[3]), "in": [], "guide": [], "out": []}
            cases.append(cur)
        else:
            conv = (lambda v: np.nan if v == "." else float(v)) if tok[0] != "guide" else int
            cur[tok[0]].append([conv(v) for v in tok[1:]])
    return cases


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_fill_hand_cases(oracle_mod, case):
    a = np.array(case["in"], dtype=np.float64)
    g = np.array(case["guide"], dtype=np.uint8) if case["guide"] else None
    got = oracle_mod.fill(a, g, case["mode"])
    exp = np.array(case["out"], dtype=np.float64)
    assert np.array_equal(np.isnan(got), np.isnan(exp))
    assert np.array_equal(got[~np.isnan(exp)], exp[~np.isnan(exp)])


def _sparse(rng, H, W, keep=0.4):
    a = rng.uniform(1, 60, size=(H, W))
    a[rng.random((H, W)) > keep] = np.nan
    a[rng.integers(0, H)] = np.nan          # at least one empty row
    return a


@pytest.mark.parametrize("mode", [0, 1])
def test_piecewise_constant_rows_are_exact(oracle_mod, mode):
    rng = np.random.default_rng(1)
    H, W = 9, 40
    full = np.zeros((H, W))
    for y in range(H):
        cuts = np.sort(rng.choice(np.arange(4, W - 4), size=3, replace=False))
        vals = rng.uniform(2, 50, size=4)
        full[y] = np.repeat(vals, np.diff(np.concatenate([[0], cuts, [W]])))
    a = full.copy()
    gaps = np.zeros_like(a, dtype=bool)
    for y in range(H):
        for x in range(1, W - 1):
            # a gap strictly inside a segment: both of its kept ends are in it
            if full[y, x - 1] == full[y, x] == full[y, x + 1] and rng.random() < 0.5:
                gaps[y, x] = True
    a[gaps] = np.nan
    g = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    got = oracle_mod.fill(a, g, mode)
    # every maximal gap run lies inside one segment, so both of its ends hold
    # the segment's constant
    assert np.array_equal(got, full)


def test_constant_guide_reduces_edge_aware_to_background(oracle_mod):
    rng = np.random.default_rng(2)
    a = _sparse(rng, 17, 23)
    flat = np.full(a.shape, 42, dtype=np.uint8)
    assert np.array_equal(oracle_mod.fill(a, flat, 1), oracle_mod.fill(a), equal_nan=True)


@pytest.mark.parametrize("mode", [0, 1])
def test_fill_keeps_kept_values_and_is_idempotent(oracle_mod, mode):
    rng = np.random.default_rng(3 + mode)
    a = _sparse(rng, 13, 31)
    g = rng.integers(0, 256, size=a.shape, dtype=np.uint8)
    f = oracle_mod.fill(a, g, mode)
    kept = ~np.isnan(a)
    assert np.array_equal(f[kept], a[kept])
    assert not np.isnan(f).any()
    assert np.array_equal(oracle_mod.fill(f, g, mode), f)
    full = rng.uniform(1, 9, size=a.shape)
    assert np.array_equal(oracle_mod.fill(full, g, mode), full)


def test_background_fill_equals_the_evaluation_module(oracle_mod):
    import torch
    from paper_1801_04720_gb300 import evaluate
    rng = np.random.default_rng(4)
    for H, W in ((7, 11), (30, 50), (3, 64)):
        a = _sparse(rng, H, W, keep=0.2)
        ev = evaluate.fill_background(torch.from_numpy(a)).numpy()
        assert np.array_equal(oracle_mod.fill(a), ev, equal_nan=True)


def test_densify_keeps_the_defined_pixels(oracle_mod):
    from paper_1801_04720_gb300 import synth
    q = synth.fronto_planes(seed=2)
    cam = q.camera
    r = oracle_mod.scene_flow(q.images(), q.flow, cam.f, cam.B, cam.cx, cam.cy, D=q.D)
    s4, motion, point, valid = oracle_mod.densify(r["s4"], q.flow, cam.f, cam.B, cam.cx, cam.cy)
    m = r["valid"] == 1
    assert m.sum() > 500 and valid.mean() > 0.95
    assert np.array_equal(s4[m], r["s4"][m])
    assert np.allclose(motion[m], r["motion"][m], rtol=0, atol=1e-12)
    assert np.allclose(point[m], r["point"][m], rtol=0, atol=1e-12)
    assert np.array_equal(np.isnan(s4[..., 0]), valid == 0)


def test_densify_closed_form_on_a_shifted_constant_scene(oracle_mod):
    H, W, d, f, B = 20, 30, 6.0, 100.0, 0.5
    rng = np.random.default_rng(5)
    u, v = 3.0, -2.0
    flow = np.zeros((H, W, 2), dtype=np.float32)
    flow[..., 0], flow[..., 1] = u, v
    s4 = np.full((H, W, 4), np.nan)
    keep = rng.random((H, W)) < 0.3
    s4[keep] = (u, v, d, d)
    cx, cy = (W - 1) / 2, (H - 1) / 2
    s4d, motion, point, valid = oracle_mod.densify(s4, flow, f, B, cx, cy)
    assert (valid == 1).all()
    assert np.allclose(motion[..., 0], u * B / d, rtol=0, atol=1e-12)
    assert np.allclose(motion[..., 1], v * B / d, rtol=0, atol=1e-12)
    assert np.allclose(motion[..., 2], 0.0, rtol=0, atol=1e-12)
    assert np.allclose(point[..., 2], f * B / d, rtol=0, atol=1e-12)
