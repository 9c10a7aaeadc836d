"""Pins for the oracle's SGM variants: the intensity-adaptive P2 of the cited
SGM (Hirschmueller 2008, cited in Sec. 3.1) and the uniqueness filter of the
winners.

* The step penalty is read off a two-pixel path whose second pixel can only
  reach the far disparity through the jump penalty, against a hand table
  (tests/golden/adaptive_p2.txt).
* Along a whole path the recurrence with per-step penalties equals the
  minimum over ALL label sequences of the path energy (exhaustive enumeration
  on tiny images), the same independent pin as for constant P2.
* A flat guide image reduces it to constant P2; flipping cost and guide
  together turns a path into its opposite; C <= L <= C + P2 still holds.
* The uniqueness verdicts of hand-worked curves (tests/golden/uniqueness.txt),
  ratio 0 keeps every winner, and a larger ratio removes a superset.
* A removed winner fails the left-right check even where the check itself
  would pass, and SGM with adaptive P2 still recovers the exact disparity
  inside textured fronto-parallel planes."""
import itertools
import os

import numpy as np
import pytest

from paper_1801_04720_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
DIRS = [(+1, 0), (-1, 0), (0, +1), (0, -1), (+1, +1), (-1, -1), (+1, -1), (-1, +1)]


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [[int(v) for v in line.split()] for line in f if line.strip() and not line.startswith("#")]


@pytest.mark.parametrize("row", _rows("adaptive_p2.txt"))
def test_step_penalty_hand_table(oracle_mod, row):
    g, P1, P2, exp = row
    # pixel 0: cost 0 at d=0 and 250 elsewhere; pixel 1: cost 0 everywhere.
    # L(1, 3) = min(C0(3), C0(2) + P1, C0(4)..., min C0 + pen) = pen (< 250).
    C = np.zeros((1, 2, 4), dtype=np.uint8)
    C[0, 0, 1:] = 250
    img = np.array([[0, g]], dtype=np.uint8)
    L = oracle_mod.path_cost(C, P1, P2, (+1, 0), img=img)
    assert L[0, 1, 3] == exp
    # the same step taken in the opposite direction (intensity step negated)
    Lb = oracle_mod.path_cost(np.ascontiguousarray(C[:, ::-1]), P1, P2, (-1, 0),
                              img=np.ascontiguousarray(img[:, ::-1]))
    assert Lb[0, 0, 3] == exp


def _path_to(p, r, W, H):
    x, y = p
    pts = [(x, y)]
    while True:
        x, y = x - r[0], y - r[1]
        if not (0 <= x < W and 0 <= y < H):
            break
        pts.append((x, y))
    return pts[::-1]


def _lun_bruteforce(C, pts, P1, pens):
    """Min energy over all label sequences along pts, per final label; pens[i]
    is the jump penalty of the step into pts[i]."""
    D = C.shape[2]
    best = np.full(D, np.iinfo(np.int64).max, dtype=np.int64)
    for seq in itertools.product(range(D), repeat=len(pts)):
        e = sum(int(C[y, x, d]) for (x, y), d in zip(pts, seq))
        for i in range(1, len(seq)):
            dd = abs(seq[i] - seq[i - 1])
            e += 0 if dd == 0 else (P1 if dd == 1 else pens[i])
        best[seq[-1]] = min(best[seq[-1]], e)
    return best


def _pen_table():
    t = {}
    for g, P1, P2, exp in _rows("adaptive_p2.txt"):
        t[(g, P1, P2)] = exp
    return t


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adaptive_path_matches_exhaustive_label_enumeration(oracle_mod, seed):
    # intensities from {0, 2, 12}: every step's |dI| (0, 2, 10 or 12) is a
    # row of the hand table, so each step's penalty is the table's
    P1, P2 = 7, 86
    table = _pen_table()
    rng = np.random.default_rng(seed)
    W, H, D = 3, 3, 4
    C = rng.integers(0, 63, size=(H, W, D), dtype=np.uint8)
    img = rng.choice(np.array([0, 2, 12], dtype=np.uint8), size=(H, W))
    assert len(np.unique(img)) > 1
    for r in DIRS:
        L = oracle_mod.path_cost(C, P1, P2, r, img=img)
        for y in range(H):
            for x in range(W):
                pts = _path_to((x, y), r, W, H)
                pens = [None] + [table[(abs(int(img[b[1], b[0]]) - int(img[a[1], a[0]])), P1, P2)]
                                 for a, b in zip(pts[:-1], pts[1:])]
                lun_p = _lun_bruteforce(C, pts, P1, pens)
                exp = lun_p if len(pts) == 1 else lun_p - _lun_bruteforce(C, pts[:-1], P1, pens[:-1]).min()
                assert np.array_equal(L[y, x], exp), (r, x, y)


@pytest.fixture(scope="module")
def scene():
    rng = np.random.default_rng(21)
    C = rng.integers(0, 63, size=(13, 17, 9), dtype=np.uint8)
    img = rng.integers(0, 256, size=(13, 17), dtype=np.uint8)
    img[4:8, 3:12] = 90       # flat patches: steps of zero keep P2
    return C, img


def test_flat_guide_reduces_to_constant_p2(oracle_mod, scene):
    C, _ = scene
    flat = np.full(C.shape[:2], 37, dtype=np.uint8)
    for mask in (0xFF, 0x0F, 0x30):
        assert np.array_equal(oracle_mod.aggregate(C, 7, 86, mask, img=flat),
                              oracle_mod.aggregate(C, 7, 86, mask))


@pytest.mark.parametrize("r", DIRS)
def test_adaptive_bounds_and_flip_symmetry(oracle_mod, scene, r):
    C, img = scene
    L = oracle_mod.path_cost(C, 7, 86, r, img=img)
    Ci = C.astype(np.int32)
    assert (L >= Ci).all() and (L <= Ci + 86).all()

    def flip(a):
        if r[0] != 0:
            a = a[:, ::-1]
        if r[1] != 0:
            a = a[::-1, :]
        return np.ascontiguousarray(a)
    Lf = oracle_mod.path_cost(flip(C), 7, 86, (-r[0], -r[1]), img=flip(img))
    assert np.array_equal(L, flip(Lf))


def test_adaptive_p2_changes_something(oracle_mod, scene):
    C, img = scene
    assert not np.array_equal(oracle_mod.aggregate(C, 7, 86, img=img), oracle_mod.aggregate(C, 7, 86))


@pytest.mark.parametrize("row", _rows("uniqueness.txt"))
def test_uniqueness_hand_curves(oracle_mod, row):
    ratio, exp, S = row[0], row[1], np.array(row[2:], dtype=np.int32)
    S3 = S.reshape(1, 1, -1)
    dint, dsub = oracle_mod.select(S3, subpixel=False)
    out = oracle_mod.uniqueness(S3, dint, dsub, ratio)
    assert (not np.isnan(out[0, 0])) == bool(exp)
    if exp:
        assert out[0, 0] == dsub[0, 0]


def test_uniqueness_zero_keeps_all_and_is_monotone(oracle_mod):
    rng = np.random.default_rng(5)
    S = rng.integers(0, 400, size=(20, 30, 24)).astype(np.int32)
    dint, dsub = oracle_mod.select(S)
    assert np.array_equal(oracle_mod.uniqueness(S, dint, dsub, 0), dsub)
    prev = np.zeros(dint.shape, dtype=bool)
    for ratio in (1, 5, 10, 25, 60):
        removed = np.isnan(oracle_mod.uniqueness(S, dint, dsub, ratio))
        assert (removed | ~prev).all() and (removed >= prev).all()
        prev = removed
    assert prev.any()


def test_removed_winner_fails_the_lr_check(oracle_mod):
    dL = np.array([[0, 1, 1, 2]], dtype=np.int16)
    dR = np.array([[0, 1, 1, 2]], dtype=np.int16)
    sub = np.array([[0.0, 1.2, np.nan, 2.0]])
    valid, disp = oracle_mod.lr_check(dL, dR, sub, 1)
    # x=1: |1 - dR[0]| = 1 keep; x=2: the check passes (|1 - dR[1]| = 0) but
    # the winner was removed; x=3: |2 - dR[1]| = 1 keep
    assert valid.tolist() == [[1, 1, 0, 1]]
    assert np.isnan(disp[0, 2]) and disp[0, 1] == 1.2


@pytest.mark.parametrize("seed", [0, 1])
def test_adaptive_p2_exact_disparity_in_plane_interiors(oracle_mod, seed):
    from test_oracle_planes import interior_mask
    q = synth.fronto_planes(seed=seed)
    r = oracle_mod.disparity(q.left_t, q.right_t, D=q.D, adaptive_p2=True, uniqueness=5)
    inner = interior_mask(q, q.surface_t, q.extra["sid_right_t"], q.gt_disp0)
    assert inner.sum() > 300
    assert np.array_equal(r["dL"][inner], q.gt_disp0[inner].astype(np.int16))
    assert (r["valid"][inner] == 1).mean() > 0.99
