"""More than two frames on the GPU (the paper's future work, Sec. 5):
the chain through K frames against the oracle (validity exact: positions are
float32 in the same order on both sides; points within 1e-5 relative), two
frames equal to the combination of Sec. 3.3, and the sequence call (each
stereo frame's SGM once) equal to per-frame SGM and per-step combinations,
and against the oracle, with the plain check and with learned confidence."""
import numpy as np
import pytest

from gpu_helpers import SUBPIXEL_ATOL, assert_nan_equal_close, to_dev, to_np
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


def _random_chain(K, H, W, seed, sigma=3.0, holes=0.15):
    rng = np.random.default_rng(seed)
    D = []
    for _ in range(K):
        d = rng.uniform(2, 40, size=(H, W)).astype(np.float32)
        d[rng.random((H, W)) < holes] = np.nan
        D.append(d)
    F = [rng.normal(0, sigma, size=(H, W, 2)).astype(np.float32) for _ in range(K - 1)]
    for f_ in F[1:]:
        m = rng.random((H, W)) < 0.3
        f_[m] = np.round(f_[m])                       # some integer flows: taps of weight zero
    return D, F


def _check_points(got_p, got_v, ref_p, ref_v):
    assert np.array_equal(got_v, ref_v)
    m = ref_v == 1
    assert m.any()
    g, r = got_p[:, m].astype(np.float64), ref_p[:, m]
    scale = np.abs(r).max(axis=-1, keepdims=True)
    assert (np.abs(g - r) <= 1e-5 * np.maximum(np.abs(r), scale)).all()
    assert np.isnan(got_p[:, ~m]).all()


@pytest.mark.parametrize("K,H,W,seed", [(2, 30, 40, 0), (3, 37, 61, 1), (5, 48, 64, 2), (8, 20, 33, 3)])
def test_chain_against_oracle(sf, oracle_mod, K, H, W, seed):
    D, F = _random_chain(K, H, W, seed)
    cam = sf.camera(100.0, 0.5, (W - 1) / 2, (H - 1) / 2)
    out = sf.sf_chain_sceneflow([to_dev(d) for d in D], [to_dev(f) for f in F], cam)
    ref_p, ref_v = oracle_mod.chain([d.astype(np.float64) for d in D], F, 100.0, 0.5, (W - 1) / 2, (H - 1) / 2)
    _check_points(to_np(out["points"]), to_np(out["valid"]), ref_p, ref_v)


def test_two_frame_chain_is_the_combination(sf):
    D, F = _random_chain(2, 41, 57, 7)
    cam = sf.camera(100.0, 0.5, 28.0, 20.0)
    d0, d1, fl = to_dev(D[0]), to_dev(D[1]), to_dev(F[0])
    ch = sf.sf_chain_sceneflow([d0, d1], [fl], cam)
    cb = sf.sf_combine_sceneflow(d0, d1, fl, cam)
    v = to_np(cb["valid"])
    assert np.array_equal(to_np(ch["valid"]), v)
    P = to_np(ch["points"])
    m = v == 1
    assert np.array_equal(P[0][m], to_np(cb["point"])[m])
    assert np.array_equal((P[1] - P[0])[m], to_np(cb["motion"])[m])


def _seq(K, seed, D=48):
    return synth.sequence(K, seed=seed, W=160, H=56, D=D, n_segments=6, disp_range=(2.0, D - 6.0))


def test_sequence_equals_per_frame_sgm_and_oracle(sf, oracle_mod):
    import torch
    K = 5
    sq = _seq(K, 3)
    c = sq.camera
    cam = sf.camera(c.f, c.B, c.cx, c.cy)
    L, R, F = [to_dev(x) for x in sq.lefts], [to_dev(x) for x in sq.rights], [to_dev(x) for x in sq.flows]
    p = sf.params(D=sq.D)
    out = sf.sf_sequence_sceneflow(L, R, F, p, cam, motion=True)
    torch.cuda.synchronize()
    for k in range(K):
        ref = sf.sf_sgm_full(L[k], R[k], p)
        assert np.array_equal(np.nan_to_num(to_np(out["disp"][k]), nan=-5.0),
                              np.nan_to_num(to_np(ref["disp"]), nan=-5.0)), k
    for k in range(K - 1):
        cb = sf.sf_combine_sceneflow(out["disp"][k], out["disp"][k + 1], F[k], cam)
        for key in ("s4", "valid", "motion"):
            a, b = to_np(out[key][k]), to_np(cb[key])
            assert np.array_equal(np.nan_to_num(a, nan=-5.0), np.nan_to_num(b, nan=-5.0)), (k, key)
    ch = sf.sf_chain_sceneflow(out["disp"], F, cam)
    assert np.array_equal(to_np(out["chain_valid"]), to_np(ch["valid"]))
    assert np.array_equal(np.nan_to_num(to_np(out["points"]), nan=-5.0),
                          np.nan_to_num(to_np(ch["points"]), nan=-5.0))
    # against the oracle: the frames' disparities, then the chain on them
    ods = [oracle_mod.disparity(sq.lefts[k], sq.rights[k], D=sq.D)["disp"] for k in range(K)]
    for k in range(K):
        assert_nan_equal_close(to_np(out["disp"][k]), ods[k], SUBPIXEL_ATOL, f"disp {k}")
    ref_p, ref_v = oracle_mod.chain(ods, sq.flows, c.f, c.B, c.cx, c.cy)
    # the GPU chain reads its own float32 disparities (within 1e-4 px of the
    # oracle's); validity depends only on which are NaN and on the flows
    _check_points(to_np(out["points"]), to_np(out["chain_valid"]), ref_p, ref_v)


def test_learned_sequence_equals_per_frame_learned(sf):
    import torch
    from paper_1801_04720_gb300 import train_confnet
    theta, meta = train_confnet.load()
    packed = sf.confnet_pack(torch.from_numpy(theta).cuda())
    thr = float(meta["threshold"])
    K = 6                                             # two groups: four passes, then two
    sq = _seq(K, 4, D=64)
    c = sq.camera
    cam = sf.camera(c.f, c.B, c.cx, c.cy)
    L, R, F = [to_dev(x) for x in sq.lefts], [to_dev(x) for x in sq.rights], [to_dev(x) for x in sq.flows]
    p = sf.params(D=sq.D)
    out = sf.sf_sequence_sceneflow(L, R, F, p, cam, packed=packed, threshold=thr)
    torch.cuda.synchronize()
    for k in range(K):
        one = sf.sf_sgm_learned(L[k], R[k], p, packed=packed, threshold=thr, features=False)
        torch.cuda.synchronize()
        assert np.array_equal(np.nan_to_num(to_np(out["disp"][k]), nan=-5.0),
                              np.nan_to_num(to_np(one["disp"]), nan=-5.0)), k


def test_sequence_arguments_are_checked(sf):
    import torch
    sq = _seq(2, 5)
    c = sq.camera
    cam = sf.camera(c.f, c.B, c.cx, c.cy)
    L = [to_dev(x) for x in sq.lefts]
    with pytest.raises(sf.SFError):       # one frame is not a sequence
        sf.sf_sequence_sceneflow(L[:1], L[:1], [], sf.params(D=sq.D), cam)
    with pytest.raises(sf.SFError):
        sf.sf_chain_sceneflow([to_dev(np.zeros((5, 5), np.float32))] * (sf.SF_MAX_FRAMES + 1),
                              [to_dev(np.zeros((5, 5, 2), np.float32))] * sf.SF_MAX_FRAMES, cam)
    torch.cuda.synchronize()
