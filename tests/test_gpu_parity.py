"""GPU parity of every C-ABI call against the CPU oracle on the same seeded
inputs: census, cost, aggregated cost, integer disparities and masks
bit-exact; subpixel disparity within 1e-4 px; scene flow within 1e-5
relative.  Sizes span several tiles with ragged tails."""
import numpy as np
import pytest

from gpu_helpers import (SUBPIXEL_ATOL, assert_nan_equal_close, assert_sceneflow_close, to_dev,
                         to_np)
from paper_1801_04720_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [(64, 48), (67, 53), (130, 41), (33, 9), (257, 20)]


@pytest.fixture(scope="module")
def sf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04720_gb300 import _lib, build
    build.build()
    _lib.load()
    return _lib


def rand_img(W, H, seed):
    return np.random.default_rng(seed).integers(0, 256, size=(H, W), dtype=np.uint8)


@pytest.mark.parametrize("W,H", SIZES)
@pytest.mark.parametrize("cw,ch", [(9, 7), (5, 5), (3, 3), (11, 5), (7, 9)])
def test_census(sf, oracle_mod, W, H, cw, ch):
    img = rand_img(W, H, W * 7 + H)
    img[H // 2, :] = 128          # flat stretches exercise the strict comparison
    got = to_np(sf.sf_census(to_dev(img), cw, ch), np.uint64)
    assert np.array_equal(got, oracle_mod.census(img, cw, ch))


@pytest.mark.parametrize("W,H", [(9, 7), (13, 7), (129, 7), (131, 10)])
def test_census_small_and_ragged(sf, oracle_mod, W, H):
    # the 9 x 7 kernel takes four columns a thread and 128 x 8 pixels a
    # block: the smallest image the window allows, a thread with one or
    # three of its columns inside, one column past a block
    img = rand_img(W, H, 3 * W + H)
    img[:, ::3] = 128
    got = to_np(sf.sf_census(to_dev(img), 9, 7), np.uint64)
    assert np.array_equal(got, oracle_mod.census(img, 9, 7))


def test_census_pitched_image(sf, oracle_mod):
    # rows of 96 bytes holding an 80-pixel image: the pitch argument is honoured
    import ctypes
    import torch
    img = rand_img(80, 30, 5)
    padded = torch.zeros((30, 96), dtype=torch.uint8, device="cuda")
    padded[:, :80] = to_dev(img)
    out = torch.empty((30, 80), dtype=torch.int64, device="cuda")
    st = sf.load().sf_census(ctypes.c_void_p(padded.data_ptr()), 80, 30, 96, 9, 7,
                             ctypes.c_void_p(out.data_ptr()), None)
    torch.cuda.synchronize()
    assert st == 0
    assert np.array_equal(to_np(out, np.uint64), oracle_mod.census(img))


@pytest.mark.parametrize("W,H", SIZES[:3])
@pytest.mark.parametrize("D", [1, 16, 37, 64, 128, 256])
@pytest.mark.parametrize("ref_is_right", [False, True])
def test_cost_volume(sf, oracle_mod, W, H, D, ref_is_right):
    q = synth.fronto_planes(W=max(W, 20), H=max(H, 12), seed=D)
    left, right = q.left_t[:H, :W].copy(), q.right_t[:H, :W].copy()
    p = sf.params(D=D)
    ref, oth = (right, left) if ref_is_right else (left, right)
    got = to_np(sf.sf_cost_volume(to_dev(ref), to_dev(oth), p, ref_is_right))
    exp = oracle_mod.cost_volume(oracle_mod.census(ref), oracle_mod.census(oth), D, ref_is_right, 62)
    assert np.array_equal(got, exp)


AGG_CASES = [
    # (W, H, D, P1, P2, mask)
    (64, 48, 16, 7, 86, 0xFF), (67, 53, 33, 7, 86, 0xFF), (130, 41, 128, 7, 86, 0xFF),
    (33, 9, 5, 7, 86, 0xFF), (40, 30, 1, 7, 86, 0xFF), (50, 20, 256, 7, 86, 0xFF),
    (45, 31, 100, 0, 0, 0xFF), (45, 31, 64, 20, 20, 0xFF), (45, 31, 64, 3, 193, 0xFF),
    (45, 31, 24, 7, 86, 0x5A), (45, 31, 24, 7, 86, 0x00),
] + [(37, 29, 40, 7, 86, 1 << r) for r in range(8)]


@pytest.mark.parametrize("staged", [False, True])
@pytest.mark.parametrize("W,H,D,P1,P2,mask", AGG_CASES)
def test_aggregate_random_cost(sf, oracle_mod, W, H, D, P1, P2, mask, staged):
    rng = np.random.default_rng(W * 1000 + D)
    C = rng.integers(0, 63, size=(H, W, D), dtype=np.uint8)
    p = sf.params(D=D, P1=P1, P2=P2, path_mask=mask)
    got = to_np(sf.sf_sgm_aggregate(to_dev(C), p, ws=None if staged else "auto"), np.uint16)
    exp = oracle_mod.aggregate(C, P1, P2, mask)
    assert np.array_equal(got.astype(np.int32), exp)


# Heights giving one band, two bands, an odd and an even band count at both
# halo widths (bands of 9 or 17 rows), so the meeting band of the merged
# launch falls on every kind of boundary.
ORDER_CASES = [(70, 7, 32), (70, 9, 32), (70, 17, 64), (70, 18, 64), (130, 41, 128), (96, 52, 48),
               (61, 35, 16), (200, 64, 256)]


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("dc,halo", [(16, 8), (16, 16), (8, 8), (8, 16)])
@pytest.mark.parametrize("W,H,D", ORDER_CASES)
def test_aggregate_every_schedule_against_oracle(sf, oracle_mod, W, H, D, dc, halo, order):
    """The fused band sweeps under each path-scheduling order and shape:
    the full aggregated cost S against the oracle, bit for bit."""
    rng = np.random.default_rng(W * 7 + H * 3 + D)
    C = rng.integers(0, 63, size=(H, W, D), dtype=np.uint8)
    p = sf.params(D=D)
    try:
        sf.sf_set_sweep_schedule(D, D, dc, halo, order)
    except sf.SFError:
        pytest.skip("shape not built for this D")
    try:
        got = to_np(sf.sf_sgm_aggregate(to_dev(C), p), np.uint16)
    finally:
        sf.sf_set_sweep_shape(D, D, 0, 0)
    assert np.array_equal(got.astype(np.int32), oracle_mod.aggregate(C, 7, 86, 0xFF))


def test_aggregate_real_cost(sf, oracle_mod):
    q = synth.fronto_planes()
    C = oracle_mod.cost_volume(oracle_mod.census(q.left_t), oracle_mod.census(q.right_t), 16)
    p = sf.params(D=16)
    got = to_np(sf.sf_sgm_aggregate(to_dev(C), p), np.uint16)
    assert np.array_equal(got.astype(np.int32), oracle_mod.aggregate(C, 7, 86, 0xFF))


@pytest.mark.parametrize("D", [1, 2, 3, 16, 33, 128, 256])
@pytest.mark.parametrize("subpixel", [True, False])
def test_select(sf, oracle_mod, D, subpixel):
    rng = np.random.default_rng(D)
    H, W = 23, 41
    S = rng.integers(0, 60, size=(H, W, D)).astype(np.int32)      # many ties
    S[::3] = rng.integers(0, 1184, size=(len(S[::3]), W, D))       # full range
    dint, dsub = sf.sf_disparity_select(to_dev(S.astype(np.int16)), subpixel)
    ei, es = oracle_mod.select(S, subpixel)
    assert np.array_equal(to_np(dint), ei)
    assert np.abs(to_np(dsub).astype(np.float64) - es).max() <= SUBPIXEL_ATOL


@pytest.mark.parametrize("tol", [0, 1, 3])
def test_lr_check(sf, oracle_mod, tol):
    rng = np.random.default_rng(tol)
    H, W, D = 30, 70, 20
    dL = rng.integers(0, D, size=(H, W)).astype(np.int16)
    dR = np.clip(dL + rng.integers(-3, 4, size=(H, W)), 0, D - 1).astype(np.int16)
    sub = (dL + rng.uniform(-0.5, 0.5, size=(H, W))).astype(np.float32)
    valid, disp = sf.sf_lr_check(to_dev(dL), to_dev(dR), to_dev(sub), tol)
    ev, ed = oracle_mod.lr_check(dL, dR, sub.astype(np.float64), tol)
    assert np.array_equal(to_np(valid), ev)
    assert_nan_equal_close(to_np(disp), ed, 0.0, "disp")


def _combine_inputs(W, H, seed):
    rng = np.random.default_rng(seed)
    D0 = rng.uniform(0.5, 120.0, size=(H, W)).astype(np.float32)
    D1 = rng.uniform(0.5, 120.0, size=(H, W)).astype(np.float32)
    D0[rng.random((H, W)) < 0.1] = np.nan
    D1[rng.random((H, W)) < 0.05] = np.nan
    D1[rng.random((H, W)) < 0.02] = 0.0
    flow = rng.normal(0, 6, size=(H, W, 2)).astype(np.float32)
    ints = rng.random((H, W)) < 0.3
    flow[ints] = np.round(flow[ints])                  # exact-tap cases
    half = rng.random((H, W)) < 0.1
    flow[half, 0] = np.round(flow[half, 0]) + 0.5
    return D0, D1, flow


@pytest.mark.parametrize("W,H", SIZES)
def test_combine(sf, oracle_mod, W, H):
    D0, D1, flow = _combine_inputs(W, H, W + H)
    cam = sf.camera(721.5, 0.54, (W - 1) / 2, (H - 1) / 2)
    out = sf.sf_combine_sceneflow(to_dev(D0), to_dev(D1), to_dev(flow), cam)
    got = {k: to_np(v) for k, v in out.items()}
    s4, motion, point, valid = oracle_mod.combine(D0.astype(np.float64), D1.astype(np.float64),
                                                  flow, float(np.float32(721.5)),
                                                  float(np.float32(0.54)), float(np.float32((W - 1) / 2)),
                                                  float(np.float32((H - 1) / 2)))
    assert valid.sum() > 0
    assert_sceneflow_close(got, s4, motion, point, valid)


@pytest.fixture(params=["fused", "staged"])
def path(sf, request):
    sf.sf_set_fused(request.param == "fused")
    yield request.param
    sf.sf_set_fused(True)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_sgm_full_planes(sf, oracle_mod, seed, path):
    q = synth.fronto_planes(seed=seed)
    p = sf.params(D=q.D)
    out = sf.sf_sgm_full(to_dev(q.left_t), to_dev(q.right_t), p)
    r = oracle_mod.disparity(q.left_t, q.right_t, D=q.D)
    assert np.array_equal(to_np(out["dL"]), r["dL"])
    assert np.array_equal(to_np(out["dR"]), r["dR"])
    assert np.array_equal(to_np(out["valid"]), r["valid"])
    assert_nan_equal_close(to_np(out["disp"]), r["disp"], SUBPIXEL_ATOL, "disp")


@pytest.mark.parametrize("W,H,D,seed", [(67, 53, 24, 5), (130, 41, 48, 6), (200, 60, 64, 7),
                                        (33, 9, 16, 8), (97, 40, 100, 9), (130, 41, 192, 10),
                                        (300, 25, 256, 11), (31, 13, 16, 12), (95, 19, 128, 13),
                                        # rows of more distances than one CTA holds (tiled cost)
                                        (1300, 20, 192, 14), (900, 18, 256, 15)])
def test_sgm_full_ragged(sf, oracle_mod, W, H, D, seed, path):
    q = synth.fronto_planes(W=W, H=H, D=D, disparities=(2, D // 3, D - 5), seed=seed)
    p = sf.params(D=D)
    out = sf.sf_sgm_full(to_dev(q.left_t), to_dev(q.right_t), p)
    r = oracle_mod.disparity(q.left_t, q.right_t, D=D)
    assert np.array_equal(to_np(out["dL"]), r["dL"])
    assert np.array_equal(to_np(out["dR"]), r["dR"])
    assert np.array_equal(to_np(out["valid"]), r["valid"])
    assert_nan_equal_close(to_np(out["disp"]), r["disp"], SUBPIXEL_ATOL, "disp")


def _scene_flow_parity(sf, oracle_mod, q, p_kw, oracle_results=None):
    W = q.shape[1]
    H = q.shape[0]
    p = sf.params(**p_kw)
    cam = sf.camera(q.camera.f, q.camera.B, q.camera.cx, q.camera.cy)
    imgs = [to_dev(im) for im in q.images()]
    out = sf.sf_scene_flow(imgs, to_dev(q.flow), p, cam)
    got = {k: (to_np(v) if v is not None else None) for k, v in out.items()}
    if oracle_results is None:
        kw = dict(D=p_kw["D"])
        r0 = oracle_mod.disparity(q.left_t, q.right_t, **kw)
        r1 = oracle_mod.disparity(q.left_t1, q.right_t1, **kw)
    else:
        r0, r1 = oracle_results
    # disparities: NaN pattern (= check) exact, values within the subpixel bound
    assert_nan_equal_close(got["D0"], r0["disp"], SUBPIXEL_ATOL, "D0")
    assert_nan_equal_close(got["D1"], r1["disp"], SUBPIXEL_ATOL, "D1")
    # validity of the end-to-end combination is an integer decision: exact
    _, _, _, valid_e2e = oracle_mod.combine(r0["disp"], r1["disp"], q.flow, q.camera.f,
                                            q.camera.B, q.camera.cx, q.camera.cy)
    assert np.array_equal(got["valid"], valid_e2e)
    # the combination kernel on the same float32 maps: 1e-5 relative
    f32 = lambda v: float(np.float32(v))
    s4, motion, point, valid = oracle_mod.combine(got["D0"].astype(np.float64),
                                                  got["D1"].astype(np.float64), q.flow,
                                                  f32(q.camera.f), f32(q.camera.B),
                                                  f32(q.camera.cx), f32(q.camera.cy))
    assert_sceneflow_close(got, s4, motion, point, valid)
    return got


@pytest.mark.parametrize("seed", [0, 1])
def test_scene_flow_planes(sf, oracle_mod, seed, path):
    q = synth.fronto_planes(seed=seed)
    got = _scene_flow_parity(sf, oracle_mod, q, dict(D=q.D))
    assert got["valid"].mean() > 0.3


def test_scene_flow_host_equals_device(sf):
    import torch
    q = synth.fronto_planes(seed=3)
    H, W = q.shape
    p = sf.params(D=q.D)
    cam = sf.camera(q.camera.f, q.camera.B, q.camera.cx, q.camera.cy)
    dev = sf.sf_scene_flow([to_dev(im) for im in q.images()], to_dev(q.flow), p, cam)
    ws = torch.empty(sf.sf_scene_flow_host_workspace_size(W, H, p), dtype=torch.uint8, device="cuda")
    host_in = [torch.from_numpy(im).pin_memory() for im in q.images()]
    flow = torch.from_numpy(q.flow).pin_memory()
    out = {"s4": torch.empty((H, W, 4)).pin_memory(), "motion": torch.empty((H, W, 3)).pin_memory(),
           "point": torch.empty((H, W, 3)).pin_memory(),
           "valid": torch.empty((H, W), dtype=torch.uint8).pin_memory()}
    sf.sf_scene_flow_host(host_in, flow, p, cam, ws, out)
    for k in ("s4", "motion", "point", "valid"):
        a, b = out[k].numpy(), to_np(dev[k])
        assert np.array_equal(np.nan_to_num(a, nan=-7.0), np.nan_to_num(b, nan=-7.0)), k


def test_status_errors_on_gpu(sf):
    import torch
    p = sf.params(D=0)
    img = torch.zeros((48, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(sf.SFError):
        sf.sf_cost_volume(img, img, p, out=torch.empty((48, 64, 1), dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()   # the context stays usable
    assert sf.sf_census(img).shape == (48, 64)


@pytest.mark.parametrize("hdc", [4, 16, 32])
@pytest.mark.parametrize("W,H,D", [(130, 41, 128), (300, 23, 96), (97, 19, 256), (64, 30, 80), (70, 17, 112)])
def test_horizontal_chunk_widths_against_oracle(sf, oracle_mod, W, H, D, hdc):
    """The horizontal paths with 16 or 32 disparities per thread (two or three
    shuffle levels in each step's minimum), or a whole warp per line pair (a
    warp-wide reduction; lanes past the depth carry padding costs): S
    bit-exact against the oracle."""
    rng = np.random.default_rng(W + H + D + hdc)
    C = rng.integers(0, 63, size=(H, W, D), dtype=np.uint8)
    sf.sf_debug_set(sf.SF_DEBUG_HLINE_DC, hdc)
    try:
        got = to_np(sf.sf_sgm_aggregate(to_dev(C), sf.params(D=D)), np.uint16)
    finally:
        sf.sf_debug_set(sf.SF_DEBUG_HLINE_DC, 0)
    assert np.array_equal(got.astype(np.int32), oracle_mod.aggregate(C, 7, 86, 0xFF))
