"""The learned scene-flow calls against the oracle, pass by pass.

sf_scene_flow_learned runs the network once over the tiles of both left
passes (t and t+1); sf_scene_flow_learned_frames with two frames runs it once
over four passes.  Here every pass of those launches is checked against the
oracle's own chain: the left-pass SGM, the features, the network forward in
float64 with the bfloat16 roundings, the acceptance rule (x - d* >= 0 and
prob >= threshold), then the combination of Sec. 3.3 (Eq. 4, 5) on the
accepted subpixel disparities.

The network's fp32 sums may differ from float64 by a bfloat16 rounding flip
now and then (a few 1e-4 in probability, see test_gpu_confnet.py), so a pixel
whose oracle probability lies within 1e-2 of the threshold may go either
way; it is excluded from the mask comparison, and so is every scene-flow
pixel that reads such a pixel (its own d0 or one of the four Eq. 5 taps of
d1).  Everything else must match: the accepted set exactly, the accepted
disparities within 1e-4 px, the scene flow within 1e-5 relative."""
import numpy as np
import pytest

from gpu_helpers import SUBPIXEL_ATOL, assert_sceneflow_close, to_dev, to_np
from oracle import confnet_oracle as co
from paper_1801_04720_gb300 import synth, train_confnet

pytestmark = pytest.mark.gpu

AMBIGUOUS = 1e-2


@pytest.fixture(scope="module")
def sf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04720_gb300 import _lib, build
    build.build()
    _lib.load()
    return _lib


@pytest.fixture(scope="module")
def net(sf):
    import torch
    theta, meta = train_confnet.load()
    packed = sf.confnet_pack(torch.from_numpy(theta).cuda())
    return theta.astype(np.float64), packed, float(meta["threshold"])


def oracle_learned_pass(oracle_mod, theta, thr, left, right, D):
    """(expected disparity map with NaN where rejected, ambiguous mask)."""
    cL, cR = oracle_mod.census(left), oracle_mod.census(right)
    C = oracle_mod.cost_volume(cL, cR, D)
    L = [oracle_mod.path_cost(C, 7, 86, r) for r in oracle_mod.DIRECTIONS]
    S = sum(L)
    feat, _ = co.features(S, L, C)
    dint, dsub = oracle_mod.select(S.astype(np.int32))
    z, _ = co.forward(theta, feat)
    prob = co.sigmoid(z)
    acc = co.learned_mask(prob, dint.astype(np.int64), thr)
    xs = np.arange(left.shape[1])[None, :]
    amb = (np.abs(prob - thr) <= AMBIGUOUS) & (xs - dint >= 0)
    return np.where(acc == 1, dsub, np.nan), amb


def sceneflow_reads_ambiguous(flow, amb0, amb1):
    """Pixels whose combination reads an ambiguous pixel: its own d0, or any
    of the four bilinear taps of d1 around x' = fl32(x + u)."""
    H, W = amb0.shape
    ys, xs = np.mgrid[0:H, 0:W]
    xp = (xs.astype(np.float32) + flow[..., 0]).astype(np.float64)
    yp = (ys.astype(np.float32) + flow[..., 1]).astype(np.float64)
    x0 = np.floor(xp).astype(np.int64)
    y0 = np.floor(yp).astype(np.int64)
    bad = amb0.copy()
    for dy in (0, 1):
        for dx in (0, 1):
            tx, ty = x0 + dx, y0 + dy
            inside = (tx >= 0) & (tx < W) & (ty >= 0) & (ty < H)
            hit = np.zeros_like(bad)
            hit[inside] = amb1[ty[inside], tx[inside]]
            bad |= hit
    return bad


def check_pass(gpu_disp, exp_disp, amb, what):
    g_acc, e_acc = ~np.isnan(gpu_disp), ~np.isnan(exp_disp)
    sure = ~amb
    diff = np.argwhere((g_acc != e_acc) & sure)
    assert diff.size == 0, f"{what}: accepted set differs at {diff[:5]}"
    both = g_acc & e_acc
    assert both.any(), f"{what}: nothing accepted"
    err = np.abs(gpu_disp[both].astype(np.float64) - exp_disp[both])
    assert err.max() <= SUBPIXEL_ATOL, f"{what}: disparity err {err.max()}"


def check_frame(oracle_mod, theta, thr, q, out):
    cam = q.camera
    e0, a0 = oracle_learned_pass(oracle_mod, theta, thr, q.left_t, q.right_t, q.D)
    e1, a1 = oracle_learned_pass(oracle_mod, theta, thr, q.left_t1, q.right_t1, q.D)
    check_pass(to_np(out["D0"]), e0, a0, "D0")
    check_pass(to_np(out["D1"]), e1, a1, "D1")
    s4, motion, point, valid = oracle_mod.combine(e0, e1, q.flow, cam.f, cam.B, cam.cx, cam.cy)
    keep = ~sceneflow_reads_ambiguous(q.flow, a0, a1)
    assert keep.mean() > 0.7
    got = {k: to_np(out[k])[keep] for k in ("s4", "motion", "point", "valid")}
    assert valid[keep].sum() > 0
    assert_sceneflow_close(got, s4[keep], motion[keep], point[keep], valid[keep])


def scenes():
    return [synth.fronto_planes(W=130, H=41, D=32, disparities=(2, 10, 27), seed=61),
            synth.automotive(seed=64, W=256, H=80, D=64, n_segments=8),
            synth.fronto_planes(W=97, H=40, D=64, disparities=(3, 20, 50), seed=63)]


@pytest.mark.parametrize("k", range(3))
def test_scene_flow_learned_every_pass_against_oracle(sf, oracle_mod, net, k):
    import torch
    theta, packed, thr = net
    q = scenes()[k]
    cam = sf.camera(q.camera.f, q.camera.B, q.camera.cx, q.camera.cy)
    out = sf.sf_scene_flow_learned([to_dev(im) for im in q.images()], to_dev(q.flow), sf.params(D=q.D), cam,
                                   packed, thr)
    torch.cuda.synchronize()
    check_frame(oracle_mod, theta, thr, q, out)


def test_two_frames_per_launch_every_pass_against_oracle(sf, oracle_mod, net):
    """Four passes in one network launch: frame 1's passes (tiles of passes 2
    and 3 of the launch) against the oracle as well as frame 0's."""
    import torch
    theta, packed, thr = net
    quads = [synth.fronto_planes(W=130, H=41, D=32, disparities=(2, 10, 27), seed=s) for s in (71, 72)]
    cam = sf.camera(quads[0].camera.f, quads[0].camera.B, quads[0].camera.cx, quads[0].camera.cy)
    sc = [([to_dev(im) for im in q.images()], to_dev(q.flow)) for q in quads]
    outs = sf.sf_scene_flow_learned_frames(sc, sf.params(D=32), cam, packed, thr)
    torch.cuda.synchronize()
    for q, o in zip(quads, outs):
        check_frame(oracle_mod, theta, thr, q, o)


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("dc,halo", [(16, 8), (8, 16)])
def test_learned_schedules_against_oracle(sf, oracle_mod, net, dc, halo, order):
    """The learned calls' own schedule table: every order and shape gives the
    oracle's result (features, network, acceptance, combination)."""
    import torch
    theta, packed, thr = net
    q = synth.automotive(seed=64, W=256, H=80, D=64, n_segments=8)
    cam = sf.camera(q.camera.f, q.camera.B, q.camera.cx, q.camera.cy)
    p = sf.params(D=q.D)
    sf.sf_set_learned_sweep_schedule(33, 64, dc, halo, order)
    try:
        # sized under the schedule in force
        ws = sf.learned_workspace(q.shape[1], q.shape[0], p, 2, "cuda")
        out = sf.sf_scene_flow_learned([to_dev(im) for im in q.images()], to_dev(q.flow), p, cam, packed, thr,
                                       ws=ws)
        torch.cuda.synchronize()
    finally:
        sf.sf_set_learned_sweep_schedule(33, 64, 0, 0, 0)
    check_frame(oracle_mod, theta, thr, q, out)
