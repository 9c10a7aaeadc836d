"""Pins for winner-take-all / subpixel refinement and the left-right check
(Sec. 3.1)."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _select_cases():
    out = []
    for line in open(os.path.join(GOLDEN, "subpixel_select.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, curve = line.split("|")
        dint, dsub = head.split()
        out.append((int(dint), float(dsub), [int(v) for v in curve.split()]))
    return out


@pytest.mark.parametrize("dint,dsub,curve", _select_cases())
def test_select_hand_cases(oracle_mod, dint, dsub, curve):
    S = np.array(curve, dtype=np.int32).reshape(1, 1, -1)
    di, ds = oracle_mod.select(S, subpixel=True)
    assert di[0, 0] == dint
    assert ds[0, 0] == dsub
    di0, ds0 = oracle_mod.select(S, subpixel=False)
    assert di0[0, 0] == dint and ds0[0, 0] == dint


def test_select_matches_first_argmin_bruteforce(oracle_mod):
    rng = np.random.default_rng(5)
    S = rng.integers(0, 40, size=(9, 11, 13), dtype=np.int32)   # many ties
    di, ds = oracle_mod.select(S, subpixel=True)
    assert np.array_equal(di, np.argmin(S, axis=2))
    off = ds - di
    assert (off > -0.5).all() and (off <= 0.5).all()


@pytest.mark.parametrize("v", [2.0, 2.1, 3.4, 3.5, 4.75, 5.9])
def test_subpixel_exact_on_sampled_parabolas(oracle_mod, v):
    # S(d) = 4 (d - v)^2 * 100 rounded is not integer in general; use
    # S(d) = A (d - v)^2 + c with A, c chosen so every sample is an integer:
    # A = 400, v given to 2 decimals -> 400 v^2 is an integer.
    d = np.arange(10)
    S = (400 * (d - v) ** 2).round().astype(np.int64)
    assert np.allclose(S, 400 * (d - v) ** 2)
    S = S.astype(np.int32).reshape(1, 1, -1)
    _, ds = oracle_mod.select(S, subpixel=True)
    assert ds[0, 0] == pytest.approx(v, abs=1e-12)


def _lr_fixture():
    rows = {}
    for line in open(os.path.join(GOLDEN, "lr_check_row.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *vals = line.split()
        rows[k] = np.array([int(v) for v in vals])
    return rows


@pytest.mark.parametrize("tol,key", [(1, "valid_tol1"), (0, "valid_tol0")])
def test_lr_check_hand_row(oracle_mod, tol, key):
    f = _lr_fixture()
    dL = f["dL"].astype(np.int16).reshape(1, -1)
    dR = f["dR"].astype(np.int16).reshape(1, -1)
    sub = dL.astype(np.float64) + 0.25
    valid, disp = oracle_mod.lr_check(dL, dR, sub, tol)
    assert np.array_equal(valid[0], f[key])
    assert np.array_equal(np.isnan(disp[0]), f[key] == 0)
    assert np.array_equal(disp[0][f[key] == 1], sub[0][f[key] == 1])


def test_lr_check_consistent_constant_maps(oracle_mod):
    d = 3
    dL = np.full((4, 20), d, dtype=np.int16)
    valid, _ = oracle_mod.lr_check(dL, dL.copy(), dL.astype(np.float64), 1)
    assert (valid[:, :d] == 0).all() and (valid[:, d:] == 1).all()
