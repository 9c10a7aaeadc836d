"""Pins for the oracle's eight-path aggregation (Sec. 3.1: "eight different
paths"; recurrence of the cited SGM with constant P1 <= P2).

The main pin is independent of the recurrence: along a path, the SGM value is
L_r(p,d) = Lun(p,d) - min_d' Lun(p-r,d'), where Lun(p,d) is the smallest path
energy sum C + sum pen over ALL label sequences ending in d at p, with
pen = 0, P1, P2 for |delta d| = 0, 1, >= 2.  The test enumerates the sequences
exhaustively on tiny images."""
import itertools

import numpy as np
import pytest

DIRS = [(+1, 0), (-1, 0), (0, +1), (0, -1), (+1, +1), (-1, -1), (+1, -1), (-1, +1)]


def _path_to(p, r, W, H):
    """Pixels from the path start to p along direction r (p last)."""
    x, y = p
    pts = [(x, y)]
    while True:
        x, y = x - r[0], y - r[1]
        if not (0 <= x < W and 0 <= y < H):
            break
        pts.append((x, y))
    return pts[::-1]


def _pen(a, b, P1, P2):
    dd = abs(a - b)
    return 0 if dd == 0 else (P1 if dd == 1 else P2)


def _lun_bruteforce(C, pts, P1, P2):
    """Min energy over all label sequences along pts, per final label."""
    D = C.shape[2]
    best = np.full(D, np.iinfo(np.int64).max, dtype=np.int64)
    for seq in itertools.product(range(D), repeat=len(pts)):
        e = sum(int(C[y, x, d]) for (x, y), d in zip(pts, seq))
        e += sum(_pen(seq[i], seq[i - 1], P1, P2) for i in range(1, len(seq)))
        best[seq[-1]] = min(best[seq[-1]], e)
    return best


@pytest.mark.parametrize("W,H,D,P1,P2,seed", [
    (4, 3, 4, 7, 86, 0), (4, 3, 4, 3, 5, 1), (3, 3, 4, 0, 9, 2), (4, 2, 3, 4, 4, 3),
    (3, 4, 4, 10, 30, 4)])
def test_path_matches_exhaustive_label_enumeration(oracle_mod, W, H, D, P1, P2, seed):
    rng = np.random.default_rng(seed)
    C = rng.integers(0, 63, size=(H, W, D), dtype=np.uint8)
    for r in DIRS:
        L = oracle_mod.path_cost(C, P1, P2, r)
        for y in range(H):
            for x in range(W):
                pts = _path_to((x, y), r, W, H)
                lun_p = _lun_bruteforce(C, pts, P1, P2)
                if len(pts) == 1:
                    exp = lun_p
                else:
                    exp = lun_p - _lun_bruteforce(C, pts[:-1], P1, P2).min()
                assert np.array_equal(L[y, x], exp), (r, x, y)


@pytest.fixture(scope="module")
def random_cost():
    rng = np.random.default_rng(11)
    return rng.integers(0, 63, size=(13, 17, 9), dtype=np.uint8)


@pytest.mark.parametrize("r", DIRS)
def test_bounds_C_le_L_le_C_plus_P2(oracle_mod, random_cost, r):
    C = random_cost.astype(np.int32)
    L = oracle_mod.path_cost(random_cost, 7, 86, r)
    assert (L >= C).all() and (L <= C + 86).all()


def test_zero_penalties_reduce_to_local_cost(oracle_mod, random_cost):
    C = random_cost.astype(np.int32)
    for r in DIRS:
        assert np.array_equal(oracle_mod.path_cost(random_cost, 0, 0, r), C)
    S = oracle_mod.aggregate(random_cost, 0, 0, 0xFF)
    assert np.array_equal(S, 8 * C)
    dint, _ = oracle_mod.select(S, subpixel=False)
    assert np.array_equal(dint, np.argmin(C, axis=2))   # local census WTA


def _flip(a, r):
    if r[0] != 0:
        a = a[:, ::-1]
    if r[1] != 0:
        a = a[::-1, :]
    return np.ascontiguousarray(a)


@pytest.mark.parametrize("r", DIRS)
def test_flip_symmetry_between_opposite_paths(oracle_mod, random_cost, r):
    # flipping the image along the axes r moves on turns direction r into -r
    L = oracle_mod.path_cost(random_cost, 7, 86, r)
    Lf = oracle_mod.path_cost(_flip(random_cost, r), 7, 86, (-r[0], -r[1]))
    assert np.array_equal(L, _flip(Lf, r))


@pytest.mark.parametrize("r", DIRS)
def test_transpose_symmetry(oracle_mod, random_cost, r):
    # swapping x and y maps direction (rx, ry) to (ry, rx)
    Ct = np.ascontiguousarray(random_cost.transpose(1, 0, 2))
    L = oracle_mod.path_cost(random_cost, 5, 40, r)
    Lt = oracle_mod.path_cost(Ct, 5, 40, (r[1], r[0]))
    assert np.array_equal(L, Lt.transpose(1, 0, 2))


def test_aggregate_is_sum_of_enabled_paths(oracle_mod, random_cost):
    total = np.zeros(random_cost.shape, dtype=np.int32)
    for i, r in enumerate(DIRS):
        Li = oracle_mod.path_cost(random_cost, 7, 86, r)
        total += Li
        S_one = oracle_mod.aggregate(random_cost, 7, 86, 1 << i)
        assert np.array_equal(S_one, Li)
    assert np.array_equal(oracle_mod.aggregate(random_cost, 7, 86, 0xFF), total)


def test_constant_cost_path_stays_constant(oracle_mod):
    # equal costs everywhere: every step adds C and the min-normalisation removes
    # nothing else, so L_r = C exactly (closed form of the recurrence)
    C = np.full((5, 6, 7), 9, dtype=np.uint8)
    for r in DIRS:
        assert (oracle_mod.path_cost(C, 7, 86, r) == 9).all()
