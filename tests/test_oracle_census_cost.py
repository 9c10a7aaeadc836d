"""Pins for the oracle's census transform and Hamming cost (Sec. 3.1: SGM with
census matching cost; window 9x7, clamped border, strict comparison)."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bit_table():
    rows = []
    for line in open(os.path.join(GOLDEN, "census_bit_index.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        dx, dy, bit = (int(v) for v in line.split())
        rows.append((dx, dy, bit))
    return rows


def test_constant_image_has_no_bits(oracle_mod):
    img = np.full((12, 15), 77, dtype=np.uint8)
    assert not oracle_mod.census(img).any()


def test_bright_isolated_pixel_sets_all_62_bits(oracle_mod):
    img = np.full((11, 13), 10, dtype=np.uint8)
    img[5, 6] = 200
    c = oracle_mod.census(img)
    assert int(c[5, 6]) == (1 << 62) - 1
    # the bright pixel is never darker than anything: every other census is 0
    c[5, 6] = 0
    assert not c.any()


@pytest.mark.parametrize("dx,dy,bit", _bit_table())
def test_bit_numbering_matches_hand_table(oracle_mod, dx, dy, bit):
    img = np.full((15, 17), 100, dtype=np.uint8)
    cy, cx = 7, 8
    img[cy + dy, cx + dx] = 3          # one strictly darker neighbour
    assert int(oracle_mod.census(img)[cy, cx]) == 1 << bit


def test_clamped_border_counts_repeated_edge_pixel(oracle_mod):
    # a dark corner pixel; census at (x=1, y=0): offsets with x+dx<=0 and y+dy<=0
    # clamp onto it: dx in [-4,-1] (4 values) x dy in [-3,0] (4 values) = 16 bits
    img = np.full((9, 12), 50, dtype=np.uint8)
    img[0, 0] = 1
    c = int(oracle_mod.census(img)[0, 1])
    assert bin(c).count("1") == 16


def test_census_invariant_under_monotone_intensity_map(oracle_mod):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 120, size=(20, 25), dtype=np.uint8)
    img2 = (img.astype(np.int32) * 2 + 7).astype(np.uint8)   # strictly increasing map
    assert np.array_equal(oracle_mod.census(img), oracle_mod.census(img2))


def test_other_window_sizes(oracle_mod):
    img = np.full((9, 9), 100, dtype=np.uint8)
    img[4, 4] = 255
    assert int(oracle_mod.census(img, 5, 5)[4, 4]) == (1 << 24) - 1
    assert int(oracle_mod.census(img, 3, 3)[4, 4]) == (1 << 8) - 1
    assert int(oracle_mod.census(img, 9, 7)[4, 4]) == (1 << 62) - 1


def _popcount_bruteforce(a, b):
    """Number of differing bits, by walking the binary string of a XOR b."""
    return bin(int(a) ^ int(b)).count("1")


def test_cost_is_hamming_distance_bruteforce(oracle_mod):
    rng = np.random.default_rng(1)
    H, W, D = 4, 11, 5
    cl = rng.integers(0, 1 << 62, size=(H, W), dtype=np.uint64)
    cr = rng.integers(0, 1 << 62, size=(H, W), dtype=np.uint64)
    C = oracle_mod.cost_volume(cl, cr, D, ref_is_right=False, cmax=62)
    CR = oracle_mod.cost_volume(cr, cl, D, ref_is_right=True, cmax=62)
    for y in range(H):
        for x in range(W):
            for d in range(D):
                exp = 62 if x - d < 0 else int(_popcount_bruteforce(cl[y, x], cr[y, x - d]))
                assert C[y, x, d] == exp
                exp = 62 if x + d > W - 1 else int(_popcount_bruteforce(cr[y, x], cl[y, x + d]))
                assert CR[y, x, d] == exp


def test_identical_images_zero_cost_at_zero_disparity(oracle_mod):
    rng = np.random.default_rng(2)
    img = rng.integers(0, 256, size=(10, 30), dtype=np.uint8)
    c = oracle_mod.census(img)
    C = oracle_mod.cost_volume(c, c, 8)
    assert not C[:, :, 0].any()


def test_shifted_image_zero_cost_at_true_disparity(oracle_mod):
    # right(x) = left(x + s): a left pixel at x matches right x - s.  Away from the
    # borders both census windows see the same pixels, so C(x, y, s) = 0.
    rng = np.random.default_rng(4)
    s = 5
    big = rng.integers(0, 256, size=(16, 60 + s), dtype=np.uint8)
    left = np.ascontiguousarray(big[:, :60])
    right = np.ascontiguousarray(big[:, s:60 + s])
    C = oracle_mod.cost_volume(oracle_mod.census(left), oracle_mod.census(right), 10)
    assert not C[3:-3, s + 4:-4, s].any()
    # and with the right image as reference, C_R(x, y, s) = 0 where x + s fits
    CR = oracle_mod.cost_volume(oracle_mod.census(right), oracle_mod.census(left), 10,
                                ref_is_right=True)
    assert not CR[3:-3, 4:60 - s - 4, s].any()
    # candidates outside the image cost cmax
    assert (C[:, 0, 1:] == 62).all()
    assert (CR[:, -1, 1:] == 62).all()
