"""The learned path's decision statistics (train_confnet.rates, calibrate,
accuracy) on hand-built maps: false-accept over the plain-removed pixels the
network decides, false-reject over the plain-kept pixels, pixels with
x - d* < 0 left to the rule, the calibration picking the smallest threshold
within the target, and the ground-truth density and error rate."""
import pytest
import torch

from paper_1801_04720_gb300 import train_confnet as tc


def _maps():
    # one row of 6 pixels; winners 0 except pixel 0, which has x - d* < 0
    prob = torch.tensor([[0.9, 0.9, 0.2, 0.8, 0.3, 0.95]])
    dint = torch.tensor([[3, 0, 0, 0, 0, 0]], dtype=torch.int16)
    valid = torch.tensor([[0, 1, 1, 0, 0, 1]], dtype=torch.uint8)   # plain check
    return prob, dint, valid


def test_rates_hand_case():
    prob, dint, valid = _maps()
    r = tc.rates([(prob, dint, valid)], threshold=0.5)
    # decided: pixels 1..5; plain-removed and decided: 3, 4 -> accepted: 3
    assert r["false_accept"] == pytest.approx(1 / 2)
    # plain-kept: 1, 2, 5 -> rejected: 2
    assert r["false_reject"] == pytest.approx(1 / 3)
    # accepted: 1, 3, 5 of 6 pixels (pixel 0 is rejected by rule)
    assert r["accepted"] == pytest.approx(3 / 6)
    assert r["plain_kept"] == pytest.approx(3 / 6)


def test_rates_pool_over_frames():
    prob, dint, valid = _maps()
    r1 = tc.rates([(prob, dint, valid)], 0.5)
    r2 = tc.rates([(prob, dint, valid), (prob, dint, valid)], 0.5)
    assert r1 == r2


def test_calibrate_smallest_threshold_within_target():
    prob, dint, valid = _maps()
    dec = [(prob, dint, valid)]
    # plain-removed decided pixels 3 (p 0.8) and 4 (p 0.3): false-accept 2/2
    # up to 0.3, 1/2 up to 0.8, 0 above; the grid runs 0.05, 0.055, ...
    t = tc.calibrate(dec, target=0.0)
    assert 0.8 < t <= 0.805 + 1e-9
    assert tc.rates(dec, t)["false_accept"] == 0.0
    assert tc.calibrate(dec, target=0.5) == pytest.approx(0.305)
    assert tc.calibrate(dec, target=1.0) == pytest.approx(0.05)


def test_accuracy_density_and_bad_pixels():
    disp = torch.tensor([[10.0, float("nan"), 20.0, 30.0]])
    gt = torch.tensor([[10.5, 5.0, 24.0, 30.0]])
    r = tc.accuracy([disp], [gt], tau=3.0)
    assert r["density"] == pytest.approx(3 / 4)
    assert r["bad_3px"] == pytest.approx(1 / 3)
