"""Learned confidence on the GPU against the oracle: features of the left
pass (bit-exact bfloat16), tensor-core inference, the training kernels
(forward, gradients, Adam) and the learned scene-flow path.

Tolerances (bf16 network, fp32 sums on the GPU, float64 in the oracle).
The fp32 sums of at most 288 products agree with float64 to about 1e-6
relative, but that is enough to move an activation across a bfloat16
rounding boundary (2^-8 relative) now and then (about 5e-4 of activations),
and a logit depends on some 2600 activations of the three hidden layers, so
most pixels carry one or two such flips, each worth |dz/da| |a| 2^-8, a few
1e-4.  So: logits within 1e-2 (1 + |z|) everywhere and 1e-3 (1 + |z|) on
average, probabilities likewise in absolute terms, gradients (sums over all
pixels) within 1e-3 of each layer's largest gradient.  Separately, inputs and
weights chosen so that every sum is exact in fp32 make the network
bit-exact up to the final sigmoid, which pins the kernel's indexing exactly."""
import numpy as np
import pytest

from gpu_helpers import to_dev, to_np
from oracle import confnet_oracle as co
from paper_1801_04720_gb300 import synth

pytestmark = pytest.mark.gpu

LAYERS = co.LAYERS


@pytest.fixture(scope="module")
def sf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04720_gb300 import _lib, build
    build.build()
    _lib.load()
    return _lib


def bf16_bits_to_float(a):
    return (np.asarray(a).view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def float_to_bf16_bits(x):
    """Exact bfloat16 values (float64) -> their 16-bit patterns as int16."""
    f = np.asarray(x, dtype=np.float32)
    assert np.array_equal(co.bf16(f), f.astype(np.float64))
    return (f.view(np.uint32) >> 16).astype(np.uint16).view(np.int16)


def oracle_left_pass(oracle_mod, left, right, D):
    cL, cR = oracle_mod.census(left), oracle_mod.census(right)
    C = oracle_mod.cost_volume(cL, cR, D)
    L = [oracle_mod.path_cost(C, 7, 86, r) for r in oracle_mod.DIRECTIONS]
    S = sum(L)
    feat, ds = co.features(S, L, C)
    dint, dsub = oracle_mod.select(S.astype(np.int32))
    return feat, ds, dint, dsub


def random_features(rng, H, W):
    return co.bf16(rng.uniform(0.0, 1.5, size=(H, W, co.F)))


# vector form of the features pass for D % 4 == 0 (one or two 128-disparity
# chunks), scalar form otherwise; the staged form (D % 32 == 0) at D = 32,
# 64, 160 and 256
SCENES = [(64, 48, 16, 0), (97, 41, 48, 1), (130, 37, 32, 2), (61, 29, 22, 3), (300, 20, 160, 4),
          (200, 16, 150, 5), (150, 33, 64, 6), (290, 19, 256, 7)]


@pytest.mark.parametrize("W,H,D,seed", SCENES)
def test_features_match_oracle(sf, oracle_mod, W, H, D, seed):
    q = synth.fronto_planes(W=W, H=H, D=D, disparities=(2, D // 3, D - 5), seed=seed)
    p = sf.params(D=D)
    out = sf.sf_sgm_learned(to_dev(q.left_t), to_dev(q.right_t), p, packed=None, features=True)
    feat_o, ds_o, dint_o, _ = oracle_left_pass(oracle_mod, q.left_t, q.right_t, D)
    assert np.array_equal(to_np(out["dint"]), dint_o)
    assert np.array_equal(ds_o, dint_o)
    got = bf16_bits_to_float(to_np(out["features"]))
    bad = np.argwhere(got != feat_o)
    assert bad.size == 0, f"features differ at {bad[:5]}: {got[tuple(bad[0])]} vs {feat_o[tuple(bad[0])]}"


def _check_close(err, what):
    """err: per-pixel error already scaled to its bound's unit."""
    assert err.max() <= 1e-2, f"max {what} error {err.max()}"
    assert err.mean() <= 1e-3, f"mean {what} error {err.mean()}"


def _check_prob(prob_gpu, prob_ref):
    _check_close(np.abs(prob_gpu.astype(np.float64) - prob_ref), "prob")


@pytest.mark.parametrize("W,H,seed", [(64, 48, 0), (56, 8, 1), (130, 37, 2), (300, 70, 3), (17, 5, 4)])
def test_infer_matches_oracle_random_features(sf, W, H, seed):
    import torch
    rng = np.random.default_rng(seed)
    theta = synth.confnet_init(seed, LAYERS)
    feat = random_features(rng, H, W)
    params = torch.from_numpy(theta).cuda()
    packed = sf.confnet_pack(params)
    out = sf.confnet_infer(packed, to_dev(float_to_bf16_bits(feat)))
    torch.cuda.synchronize()
    z, _ = co.forward(theta.astype(np.float64), feat)
    _check_prob(to_np(out["prob"]), co.sigmoid(z))


def _exact_params(rng):
    """Sparse weights that are small multiples of powers of two: every partial
    sum of the network is a multiple of 2^-15 below 2^9, exact in fp32."""
    theta = np.zeros(co.param_count())
    for li, (w, b) in enumerate(co.split_params(theta)):
        co_, ci = w.shape[0], w.shape[3]
        for o in range(co_):
            for _ in range(3 if li else 4):
                ky, kx, c = rng.integers(0, 3), rng.integers(0, 3), rng.integers(0, ci)
                w[o, ky, kx, c] = rng.choice([-0.5, -0.25, 0.25, 0.5])
        b[:] = rng.integers(-4, 5, size=b.shape) / 16.0
    return theta


@pytest.mark.parametrize("W,H,seed", [(64, 48, 0), (130, 37, 1), (200, 90, 2)])
def test_infer_bit_exact_on_exact_arithmetic(sf, W, H, seed):
    import torch
    rng = np.random.default_rng(100 + seed)
    theta = _exact_params(rng)
    feat = rng.integers(0, 16, size=(H, W, co.F)) / 8.0
    packed = sf.confnet_pack(torch.from_numpy(theta.astype(np.float32)).cuda())
    out = sf.confnet_infer(packed, to_dev(float_to_bf16_bits(feat)))
    torch.cuda.synchronize()
    z, acts = co.forward(theta, feat)
    for a in acts[1:]:
        assert np.abs(a).max() < 2 ** 9
    # the logit is exact on both sides; only the fp32 sigmoid differs
    assert np.abs(to_np(out["prob"]).astype(np.float64) - co.sigmoid(z)).max() <= 1e-6


def test_infer_on_oracle_features_with_biases_and_mask(sf, oracle_mod):
    import torch
    q = synth.fronto_planes(W=130, H=37, D=32, disparities=(2, 10, 27), seed=7)
    feat, ds, dint, dsub = oracle_left_pass(oracle_mod, q.left_t, q.right_t, 32)
    rng = np.random.default_rng(8)
    theta = synth.confnet_init(8, LAYERS).astype(np.float64)
    for (w, b) in co.split_params(theta):
        b[:] = rng.normal(0, 0.1, size=b.shape)
    theta32 = theta.astype(np.float32)
    packed = sf.confnet_pack(torch.from_numpy(theta32).cuda())
    dsub32 = dsub.astype(np.float32)
    out = sf.confnet_infer(packed, to_dev(float_to_bf16_bits(feat)), to_dev(dint), to_dev(dsub32),
                           threshold=0.5)
    torch.cuda.synchronize()
    z, _ = co.forward(theta32.astype(np.float64), feat)
    pr = co.sigmoid(z)
    pg = to_np(out["prob"])
    _check_prob(pg, pr)
    # the acceptance rule, decided on the GPU's own probability
    exp_valid = co.learned_mask(pg.astype(np.float64), dint.astype(np.int64), 0.5)
    assert np.array_equal(to_np(out["valid"]), exp_valid)
    disp = to_np(out["disp"])
    m = exp_valid == 1
    assert np.array_equal(disp[m], dsub32[m])
    assert np.isnan(disp[~m]).all()
    # and, away from the threshold, on the oracle's probability
    far = np.abs(pr - 0.5) > 1e-2
    assert np.array_equal(exp_valid[far], co.learned_mask(pr, dint.astype(np.int64), 0.5)[far])


def _batch(rng, B, H, W, theta_seed):
    feats = np.stack([random_features(rng, H, W) for _ in range(B)])
    labels = rng.integers(0, 2, size=(B, H, W)).astype(np.uint8)
    labels[:, 0, :3] = 255
    theta = synth.confnet_init(theta_seed, LAYERS).astype(np.float64)
    for (w, b) in co.split_params(theta):
        b[:] = rng.normal(0, 0.05, size=b.shape)
    return feats, labels, theta.astype(np.float32)


def test_training_forward_matches_oracle(sf):
    import torch
    rng = np.random.default_rng(11)
    feats, _, theta = _batch(rng, 2, 23, 37, 11)
    params = torch.from_numpy(theta).cuda()
    fb = to_dev(np.stack([float_to_bf16_bits(f) for f in feats]))
    logits = torch.empty((2, 23, 37), dtype=torch.float32, device="cuda")
    hp = sf.hparams(lr=0.0)
    sf.confnet_train_step(params, None, None, fb, None, hp, logits=logits)
    torch.cuda.synchronize()
    for b in range(2):
        z, _ = co.forward(theta.astype(np.float64), feats[b])
        _check_close(np.abs(to_np(logits[b]).astype(np.float64) - z) / (1.0 + np.abs(z)), "logit")


@pytest.mark.parametrize("B,H,W,w_neg", [(2, 21, 34, 1.0), (3, 16, 16, 4.0), (1, 9, 70, 2.5)])
def test_training_gradients_match_oracle(sf, B, H, W, w_neg):
    import torch
    rng = np.random.default_rng(B * 100 + W)
    feats, labels, theta = _batch(rng, B, H, W, W)
    params = torch.from_numpy(theta.copy()).cuda()
    fb = to_dev(np.stack([float_to_bf16_bits(f) for f in feats]))
    grad = torch.empty(co.param_count(), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    hp = sf.hparams(lr=0.0, w_neg=w_neg)      # lr 0: the step leaves the parameters unchanged
    sf.confnet_train_step(params, m, v, fb, to_dev(labels), hp, grad=grad, loss=loss)
    torch.cuda.synchronize()
    L, g = co.loss_and_grads(theta.astype(np.float64), feats, labels, w_neg)
    assert abs(float(loss.item()) - L) <= 1e-5 * max(1.0, abs(L))
    gg = to_np(grad).astype(np.float64)
    o = 0
    for ci, c_o in LAYERS:
        n = 9 * ci * c_o + c_o
        ref, got = g[o:o + n], gg[o:o + n]
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-3 * scale + 1e-9, (ci, c_o, np.abs(got - ref).max(), scale)
        o += n
    assert np.array_equal(to_np(params), theta)


def test_adam_matches_oracle(sf):
    import torch
    rng = np.random.default_rng(5)
    n = co.param_count()
    theta = rng.normal(0, 0.1, n).astype(np.float32)
    m = rng.normal(0, 1e-3, n).astype(np.float32)
    v = rng.uniform(0, 1e-5, n).astype(np.float32)
    g = rng.normal(0, 1e-2, n).astype(np.float32)
    hp = sf.hparams(lr=2e-3, beta1=0.9, beta2=0.999, eps=1e-8, step=7)
    tt, mt, vt = (torch.from_numpy(a.copy()).cuda() for a in (theta, m, v))
    sf.confnet_adam(tt, mt, vt, torch.from_numpy(g).cuda(), hp)
    torch.cuda.synchronize()
    # the oracle at the fp32 hyperparameters the kernel receives
    f = lambda x: float(np.float32(x))
    b1, b2 = f(0.9), f(0.999)
    t2, m2, v2 = co.adam(theta.astype(np.float64), m.astype(np.float64), v.astype(np.float64),
                         g.astype(np.float64), 7, f(2e-3), b1, b2, f(1e-8))
    # a few fp32 roundings of terms of these sizes
    u = 2.0 ** -22
    assert (np.abs(to_np(mt) - m2) <= u * (b1 * np.abs(m) + (1 - b1) * np.abs(g))).all()
    assert (np.abs(to_np(vt) - v2) <= u * (b2 * v + (1 - b2) * g.astype(np.float64) ** 2)).all()
    step = np.abs(t2 - theta)
    assert (np.abs(to_np(tt).astype(np.float64) - t2) <= u * np.abs(theta) + 1e-5 * step).all()


def test_training_reduces_the_loss(sf):
    import torch
    rng = np.random.default_rng(21)
    feats, labels, theta = _batch(rng, 4, 32, 32, 21)
    # a learnable rule: accept where feature 0 is small
    labels = (feats[..., 0] < 0.75).astype(np.uint8)
    params = torch.from_numpy(theta).cuda()
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    fb = to_dev(np.stack([float_to_bf16_bits(f) for f in feats]))
    lab = to_dev(labels)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    ws = sf.confnet_train_workspace(4, 32, 32, "cuda")
    losses = []
    for step in range(1, 61):
        sf.confnet_train_step(params, m, v, fb, lab, sf.hparams(lr=3e-3, step=step), ws=ws, loss=loss)
        losses.append(float(loss.item()))
    assert losses[-1] < 0.5 * losses[0], losses[::10]


def test_scene_flow_learned_uses_the_plain_disparities(sf):
    """Accepted pixels carry exactly the plain path's subpixel disparity, and
    the combination equals sf_combine_sceneflow on those maps."""
    import torch
    q = synth.fronto_planes(W=96, H=64, D=16, seed=3)
    H, W = q.shape
    theta = synth.confnet_init(3, LAYERS)
    params = torch.from_numpy(theta).cuda()
    packed = sf.confnet_pack(params)
    imgs = [to_dev(im) for im in q.images()]
    cam = sf.camera(q.camera.f, q.camera.B, q.camera.cx, q.camera.cy)
    p = sf.params(D=q.D)
    out = sf.sf_scene_flow_learned(imgs, to_dev(q.flow), p, cam, packed, 0.3)
    # plain subpixel winners everywhere x - d >= 0 (tolerance wide open)
    p_all = sf.params(D=q.D, lr_tol=10000)
    for D_l, (l, r) in ((out["D0"], (imgs[0], imgs[1])), (out["D1"], (imgs[2], imgs[3]))):
        plain = sf.sf_sgm_full(l, r, p_all)
        a, b = to_np(D_l), to_np(plain["disp"])
        acc = ~np.isnan(a)
        assert acc.any()
        assert np.array_equal(a[acc], b[acc])
    ref = sf.sf_combine_sceneflow(out["D0"], out["D1"], to_dev(q.flow), cam)
    torch.cuda.synchronize()
    for k in ("s4", "valid"):
        x, y = to_np(out[k]), to_np(ref[k])
        assert np.array_equal(np.nan_to_num(x, nan=-7.0), np.nan_to_num(y, nan=-7.0)), k


def test_learned_path_rejects_partial_path_masks(sf):
    import torch
    q = synth.fronto_planes(seed=0)
    p = sf.params(D=16, path_mask=0x0F)
    with pytest.raises(sf.SFError):
        sf.sf_sgm_learned(to_dev(q.left_t), to_dev(q.right_t), p, packed=None)
    torch.cuda.synchronize()


def test_two_frames_per_launch_equal_single_frames(sf):
    import torch
    theta = synth.confnet_init(5, LAYERS)
    packed = sf.confnet_pack(torch.from_numpy(theta).cuda())
    quads = [synth.fronto_planes(W=130, H=41, D=32, disparities=(2, 10, 27), seed=s) for s in (31, 32)]
    cam = sf.camera(quads[0].camera.f, quads[0].camera.B, quads[0].camera.cx, quads[0].camera.cy)
    p = sf.params(D=32)
    scenes = [([to_dev(im) for im in q.images()], to_dev(q.flow)) for q in quads]
    both = sf.sf_scene_flow_learned_frames(scenes, p, cam, packed, 0.4)
    torch.cuda.synchronize()
    for (imgs, flow), o in zip(scenes, both):
        one = sf.sf_scene_flow_learned(imgs, flow, p, cam, packed, 0.4)
        torch.cuda.synchronize()
        for k in ("s4", "motion", "point", "valid", "D0", "D1"):
            a, b = to_np(o[k]), to_np(one[k])
            assert np.array_equal(np.nan_to_num(a, nan=-3.0), np.nan_to_num(b, nan=-3.0)), k
