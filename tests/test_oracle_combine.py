"""Pins for the oracle's combination step (Sec. 3.3, Eq. 3-5) and its
back-projection Z = fB/d."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    grid, cases, full = [], [], []
    for line in open(os.path.join(GOLDEN, "bilinear_eq5.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *vals = line.split()
        if k == "grid":
            grid.append([float(v) for v in vals])
        elif k == "case":
            cases.append([float(v) for v in vals])
        elif k == "full":
            full.append([float(v) for v in vals])
    return np.array(grid), cases, full


def _run_single(oracle_mod, D1, x, y, u, v, d0=10.0, cam=(100.0, 0.5, 2.0, 1.5)):
    H, W = D1.shape
    D0 = np.full((H, W), d0)
    flow = np.zeros((H, W, 2), dtype=np.float32)
    flow[y, x] = (u, v)
    return oracle_mod.combine(D0, D1, flow, *cam)


def test_eq5_hand_cases(oracle_mod):
    D1, cases, _ = _golden()
    for x, y, u, v, valid, d1 in cases:
        x, y = int(x), int(y)
        s4, motion, point, ok = _run_single(oracle_mod, D1, x, y, u, v)
        assert ok[y, x] == int(valid), (x, y, u, v)
        if valid:
            assert s4[y, x, 3] == pytest.approx(d1, abs=1e-12)
            assert s4[y, x, 0] == u and s4[y, x, 1] == v and s4[y, x, 2] == 10.0
        else:
            assert np.isnan(s4[y, x]).all() and np.isnan(motion[y, x]).all()


def test_backprojection_hand_case(oracle_mod):
    D1, _, full = _golden()
    for x, y, s_u, s_v, s_d0, s_d1, mx, my, mz in full:
        x, y = int(x), int(y)
        s4, motion, point, ok = _run_single(oracle_mod, D1, x, y, s_u, s_v)
        assert ok[y, x] == 1
        assert np.allclose(s4[y, x], [s_u, s_v, s_d0, s_d1], rtol=0, atol=1e-12)
        assert np.allclose(motion[y, x], [mx, my, mz], rtol=0, atol=1e-12)
        assert np.allclose(point[y, x], [-0.05, -0.025, 5.0], rtol=0, atol=1e-12)


def test_integer_shift_constant_depth_closed_form(oracle_mod):
    # constant disparity d, integer flow (u, v): the point keeps its depth and
    # moves by (uB/d, vB/d, 0); Z = fB/d.  Pixels shifted out of the image are
    # undefined (Eq. 4).
    H, W, d = 12, 20, 4.0
    f, B = 100.0, 0.5
    cx, cy = (W - 1) / 2, (H - 1) / 2
    rng = np.random.default_rng(0)
    flow = rng.integers(-3, 4, size=(H, W, 2)).astype(np.float32)
    D = np.full((H, W), d)
    s4, motion, point, ok = oracle_mod.combine(D, D, flow, f, B, cx, cy)
    ys, xs = np.mgrid[0:H, 0:W]
    inside = ((xs + flow[..., 0] >= 0) & (xs + flow[..., 0] <= W - 1) &
              (ys + flow[..., 1] >= 0) & (ys + flow[..., 1] <= H - 1))
    assert np.array_equal(ok == 1, inside)
    m = inside
    assert np.allclose(motion[m, 0], flow[m, 0] * B / d, atol=1e-13)
    assert np.allclose(motion[m, 1], flow[m, 1] * B / d, atol=1e-13)
    assert np.allclose(motion[m, 2], 0.0, atol=1e-13)
    assert np.allclose(point[m, 2], f * B / d, atol=1e-13)
    assert np.allclose(point[m, 0], (xs[m] - cx) * B / d, atol=1e-13)


def test_bilinear_reproduces_bilinear_functions(oracle_mod):
    # Eq. 5 is exact for D1(x, y) = a + b x + c y + e x y (the bilinear family)
    H, W = 10, 14
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    a, b, c, e = 20.0, 0.5, -0.75, 0.03
    D1 = a + b * xs + c * ys + e * xs * ys
    rng = np.random.default_rng(1)
    flow = rng.uniform(-2.5, 2.5, size=(H, W, 2)).astype(np.float32)
    D0 = np.full((H, W), 7.0)
    s4, _, _, ok = oracle_mod.combine(D0, D1, flow, 100.0, 0.5, 6.5, 4.5)
    xp = (xs.astype(np.float32) + flow[..., 0]).astype(np.float64)
    yp = (ys.astype(np.float32) + flow[..., 1]).astype(np.float64)
    exp = a + b * xp + c * yp + e * xp * yp
    m = ok == 1
    assert m.sum() > 50
    assert np.allclose(s4[m, 3], exp[m], rtol=0, atol=1e-12)


def test_invalid_taps_and_disparity_rules(oracle_mod):
    H, W = 6, 6
    D1 = np.full((H, W), 5.0)
    D1[2, 3] = np.nan            # removed by the consistency check
    D1[4, 4] = 0.0               # zero disparity cannot be back-projected
    D0 = np.full((H, W), 5.0)
    D0[0, 0] = np.nan
    flow = np.zeros((H, W, 2), dtype=np.float32)
    flow[1, 2] = (0.5, 0.5)      # taps (2,1) (3,1) (2,2) (3,2): (3,2) is nan -> undefined
    flow[1, 1] = (0.0, 0.5)      # taps (1,1) (1,2) only: fine
    flow[3, 3] = (1.0, 1.0)      # lands on (4,4) which has d=0 -> undefined
    _, _, _, ok = oracle_mod.combine(D0, D1, flow, 100.0, 0.5, 2.5, 2.5)
    assert ok[1, 2] == 0 and ok[1, 1] == 1 and ok[3, 3] == 0
    assert ok[0, 0] == 0         # D0 invalid
    assert ok[2, 3] == 0         # flow 0 lands on its own D1 sample, which is nan
    assert ok[4, 4] == 0 and ok[5, 5] == 1
