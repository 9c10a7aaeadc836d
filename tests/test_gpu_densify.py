"""Densification on the GPU against the oracle (the paper's future work,
Sec. 5; Table 1's dense rows are the benchmark's fill of a sparse result):
the filled maps bit-exact in both modes (a fill copies kept float32 values),
the dense scene flow's (u, v, d0, d1) and validity exact and its
back-projection within 1e-5 relative, on maps with empty rows, ragged row
lengths (not multiples of the 32-pixel warp chunk), single rows and columns,
and the real sparse output of the 1242 x 375 automotive frame."""
import numpy as np
import pytest

from gpu_helpers import assert_sceneflow_close, to_dev, to_np
from paper_1801_04720_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04720_gb300 import _lib, build
    build.build()
    _lib.load()
    return _lib


def _sparse(rng, H, W, keep):
    a = rng.uniform(1, 120, size=(H, W)).astype(np.float32)
    a[rng.random((H, W)) > keep] = np.nan
    if H > 2:
        a[rng.integers(0, H, size=max(1, H // 5))] = np.nan      # empty rows
    return a


SIZES = [(1, 1), (1, 37), (29, 1), (7, 31), (13, 32), (17, 33), (40, 100), (75, 1242), (33, 2048)]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("H,W", SIZES)
@pytest.mark.parametrize("keep", [0.02, 0.5, 0.97])
def test_fill_against_oracle(sf, oracle_mod, H, W, keep, mode):
    rng = np.random.default_rng(H * 131 + W + int(keep * 100) + mode)
    a = _sparse(rng, H, W, keep)
    g = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    g[:, : W // 3] = 40                                        # flat part: ties
    got = to_np(sf.sf_fill_disparity(to_dev(a), to_dev(g), mode))
    exp = oracle_mod.fill(a.astype(np.float64), g, mode)
    assert np.array_equal(np.isnan(got), np.isnan(exp))
    m = ~np.isnan(exp)
    assert np.array_equal(got[m].astype(np.float64), exp[m])


def test_fill_of_nothing_kept_stays_missing(sf):
    a = np.full((9, 40), np.nan, dtype=np.float32)
    assert np.isnan(to_np(sf.sf_fill_disparity(to_dev(a)))).all()


@pytest.fixture(scope="module")
def frame(sf, oracle_mod):
    q = synth.automotive(seed=3)
    c = q.camera
    cam = sf.camera(c.f, c.B, c.cx, c.cy)
    out = sf.sf_scene_flow([to_dev(im) for im in q.images()], to_dev(q.flow), sf.params(D=q.D), cam)
    return q, cam, out


@pytest.mark.parametrize("mode", [0, 1])
def test_densify_automotive_frame_against_oracle(sf, oracle_mod, frame, mode):
    q, cam, out = frame
    c = q.camera
    s4 = to_np(out["s4"])
    assert np.isnan(s4[..., 2]).mean() > 0.3                  # sparse to begin with
    got = sf.sf_densify_sceneflow(out["s4"], to_dev(q.flow), cam, guide=to_dev(q.left_t), mode=mode)
    s4o, motion, point, valid = oracle_mod.densify(s4.astype(np.float64), q.flow, c.f, c.B, c.cx, c.cy,
                                                   guide=q.left_t, mode=mode)
    g = {k: to_np(got[k]) for k in ("s4", "motion", "point", "valid")}
    assert np.array_equal(g["valid"], valid)
    assert valid.mean() > 0.99
    m = valid == 1
    assert np.array_equal(g["s4"][m].astype(np.float64), s4o[m])        # copies of float32 values
    assert_sceneflow_close(g, s4o, motion, point, valid)


def test_densify_against_oracle_sparse_synthetic(sf, oracle_mod):
    rng = np.random.default_rng(9)
    H, W = 45, 77
    s4 = np.full((H, W, 4), np.nan, dtype=np.float32)
    keep = rng.random((H, W)) < 0.3
    s4[keep, 2] = rng.uniform(1, 60, size=keep.sum())
    s4[keep, 3] = rng.uniform(1, 60, size=keep.sum())
    s4[3, :, 2:] = np.nan                                      # an empty row in both maps
    s4[keep & (rng.random((H, W)) < 0.05), 3] = -1.0          # a non-positive d1: invalid after the fill
    flow = rng.normal(0, 3, size=(H, W, 2)).astype(np.float32)
    cam = sf.camera(100.0, 0.5, (W - 1) / 2, (H - 1) / 2)
    got = sf.sf_densify_sceneflow(to_dev(s4), to_dev(flow), cam)
    s4o, motion, point, valid = oracle_mod.densify(s4.astype(np.float64), flow, 100.0, 0.5, (W - 1) / 2,
                                                   (H - 1) / 2)
    g = {k: to_np(got[k]) for k in ("s4", "motion", "point", "valid")}
    assert np.array_equal(g["valid"], valid)
    assert 0.5 < valid.mean() < 1.0
    assert_sceneflow_close(g, s4o, motion, point, valid)


def test_densify_arguments_are_checked(sf):
    import torch
    a = torch.zeros((10, 20), dtype=torch.float32, device="cuda")
    with pytest.raises(sf.SFError):
        sf.sf_fill_disparity(a, out=a)                 # in place
    with pytest.raises(sf.SFError):
        sf.sf_fill_disparity(a, mode=1)                # edge-aware needs the guide
    with pytest.raises(sf.SFError):
        sf.sf_fill_disparity(a, mode=2)
    s4 = torch.zeros((10, 20, 4), dtype=torch.float32, device="cuda")
    flow = torch.zeros((10, 20, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(sf.SFError):
        sf.sf_densify_sceneflow(s4, flow, sf.camera(100.0, 0.5, 9.5, 4.5), out={"s4": s4, "motion": None,
                                                                              "point": None, "valid": None})
