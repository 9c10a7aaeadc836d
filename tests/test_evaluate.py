"""KITTI-style accuracy figures (evaluate.py) on hand-built results: each
outlier rule, the combination into SF, density, and pixels without ground
truth."""
import math

import pytest
import torch

from paper_1801_04720_gb300 import evaluate as ev


def _scene(H=2, W=5):
    gt0 = torch.full((H, W), 40.0)
    gt1 = torch.full((H, W), 38.0)
    gtf = torch.zeros((H, W, 2))
    gtf[..., 0] = 10.0
    s4 = torch.stack([gtf[..., 0], gtf[..., 1], gt0, gt1], dim=-1).clone()
    valid = torch.ones((H, W), dtype=torch.uint8)
    return s4, valid, gt0, gt1, gtf


def test_exact_results_have_no_outliers():
    s4, valid, gt0, gt1, gtf = _scene()
    r = ev.scene_flow_accuracy(s4, valid, gt0, gt1, gtf)
    assert r == {"density": 1.0, "D1": 0.0, "D2": 0.0, "Fl": 0.0, "SF": 0.0}


def test_both_thresholds_must_be_exceeded():
    # true disparity 40: 5 % is 2 px, so the 3 px rule decides; true 100:
    # 5 % is 5 px, so an error of 4 px is not an outlier
    err = torch.tensor([2.9, 3.1, 4.0, 6.0])
    mag = torch.tensor([40.0, 40.0, 100.0, 100.0])
    assert ev.outliers(err, mag).tolist() == [False, True, False, True]


def test_each_component_and_their_union():
    s4, valid, gt0, gt1, gtf = _scene()
    s4[0, 0, 2] += 5.0          # D1 outlier
    s4[0, 1, 3] -= 4.0          # D2 outlier
    s4[0, 2, 1] += 3.5          # Fl outlier (|(0, 3.5)| = 3.5 > max(3, 0.5))
    s4[0, 3, 2] += 5.0          # D1 and D2 at one pixel: one SF outlier
    s4[0, 3, 3] += 5.0
    s4[1, 0, 2] += 2.0          # below both thresholds
    r = ev.scene_flow_accuracy(s4, valid, gt0, gt1, gtf)
    assert r["D1"] == pytest.approx(2 / 10)
    assert r["D2"] == pytest.approx(2 / 10)
    assert r["Fl"] == pytest.approx(1 / 10)
    assert r["SF"] == pytest.approx(4 / 10)


def test_rates_over_kept_pixels_and_density():
    s4, valid, gt0, gt1, gtf = _scene()
    s4[0, 0, 2] = float("nan")   # a dropped pixel carries NaN; not evaluated
    valid[0, 0] = 0
    s4[1, 4, 2] += 10.0
    valid[1, 3] = 0
    r = ev.scene_flow_accuracy(s4, valid, gt0, gt1, gtf)
    assert r["density"] == pytest.approx(8 / 10)
    assert r["D1"] == pytest.approx(1 / 8)


def test_pixels_without_ground_truth_are_left_out():
    s4, valid, gt0, gt1, gtf = _scene()
    gt1[1, :] = math.inf
    s4[1, 2, 3] += 50.0          # would be an outlier, but has no ground truth
    r = ev.scene_flow_accuracy(s4, valid, gt0, gt1, gtf)
    assert r["density"] == 1.0
    assert r["D2"] == 0.0 and r["SF"] == 0.0


def test_nothing_kept():
    s4, valid, gt0, gt1, gtf = _scene()
    r = ev.scene_flow_accuracy(s4, torch.zeros_like(valid), gt0, gt1, gtf)
    assert r == {"density": 0.0, "D1": 0.0, "D2": 0.0, "Fl": 0.0, "SF": 0.0}


def test_fill_background_rows_hand_case():
    nan = float("nan")
    a = torch.tensor([[nan, 5.0, nan, nan, 9.0, 7.0, nan],
                      [1.0, nan, 3.0, nan, nan, nan, nan]])
    got = ev.fill_background(a)
    # row 0: leading run takes 5; the run between 5 and 9 takes min = 5;
    # the trailing run takes 7.  Row 1: 1 | min(1, 3) | 3 | trailing 3s
    assert got.tolist() == [[5.0, 5.0, 5.0, 5.0, 9.0, 7.0, 7.0],
                            [1.0, 1.0, 3.0, 3.0, 3.0, 3.0, 3.0]]


def test_fill_background_empty_rows_take_columns():
    nan = float("nan")
    a = torch.tensor([[nan, nan, nan],
                      [2.0, nan, 8.0],
                      [nan, nan, nan],
                      [6.0, 4.0, nan]])
    got = ev.fill_background(a)
    # rows 1 and 3 fill along the row first: [2, 2, 8] and [6, 4, 4]; rows 0
    # and 2 have nothing and take their columns of that row-filled map: row 0
    # from the row below, row 2 the smaller of its neighbours above and below
    assert got[1].tolist() == [2.0, 2.0, 8.0]
    assert got[3].tolist() == [6.0, 4.0, 4.0]
    assert got[0].tolist() == [2.0, 2.0, 8.0]
    assert got[2].tolist() == [2.0, 2.0, 4.0]


def test_fill_background_all_missing_stays_missing():
    a = torch.full((2, 3), float("nan"))
    assert torch.isnan(ev.fill_background(a)).all()


def test_dense_accuracy_uses_input_flow_and_filled_disparities():
    s4, valid, gt0, gt1, gtf = _scene()
    flow = gtf.clone()
    s4[0, 1:4, :] = float("nan")          # a gap in row 0
    s4[0, 0, 2] = 38.0                    # left neighbour of the gap (error 2 px)
    r = ev.scene_flow_accuracy_dense(s4, flow, gt0, gt1, gtf)
    assert r["density"] == 1.0
    # the gap takes min(38, 40) = 38 for d0: errors of 2 px, not outliers
    assert r["D1"] == 0.0 and r["SF"] == 0.0
    s4[0, 0, 2] = 30.0                    # now the fill is 10 px off on 4 pixels
    r = ev.scene_flow_accuracy_dense(s4, flow, gt0, gt1, gtf)
    assert r["D1"] == pytest.approx(4 / 10)
