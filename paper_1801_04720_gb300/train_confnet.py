"""Training, calibration and evaluation of the learned confidence network.

Two scene recipes feed it: the fronto-parallel plane recipe and the
automotive recipe (slanted moving segments over a ground plane and a far
wall), both at 1242x375, D = 128; from the automotive recipe both stereo
pairs of a quadruple are used.  Labels come from the plain method itself: a pixel of the left pass is a
positive when the left-right check (Sec. 3.1, tolerance 1 px) keeps it and a
negative when the check removes it; pixels with x - d* < 0 are left out (the
learned path rejects them by rule).  Every step runs through libsf: the
plain stereo pass makes the labels, the learned pass the features, the
training kernels the optimisation, the tensor-core kernel the inference.
PyTorch only holds device memory and batches crops.

    python -m paper_1801_04720_gb300.train_confnet [--scenes 2000] [--out FILE]

writes the fp32 parameters, the calibrated threshold and the evaluation to
an .npz file (default: confnet_weights.npz beside this module)."""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "confnet_weights.npz")
LAYERS = [(8, 32), (32, 32), (32, 32), (32, 1)]
# plane recipe (one pair per seed)
TRAIN_SEEDS = range(0, 2000)
CALIB_SEEDS = range(5000, 5100)
EVAL_SEEDS = range(10000, 10200)
# automotive recipe (two pairs per seed); disjoint from the seeds the bench renders
AUTO_TRAIN_SEEDS = range(20000, 20600)
AUTO_CALIB_SEEDS = range(25000, 25040)
AUTO_EVAL_SEEDS = range(30000, 30050)


def _render(args):
    from paper_1801_04720_gb300 import synth
    seed, W, H, D, recipe = args
    if recipe == "automotive":
        q = synth.automotive(seed=seed, W=W, H=H, D=D)
        return [(q.left_t, q.right_t), (q.left_t1, q.right_t1)]
    q = synth.confidence_recipe(seed, W=W, H=H, D=D)
    return [(q.left_t, q.right_t)]


def render_pairs(seeds, W, H, D, recipe="planes", workers=None):
    """Stereo pairs of a recipe ("planes": the left/right images at t;
    "automotive": both pairs of each quadruple), rendered on the host in
    spawned worker processes."""
    workers = workers or min(16, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        per_seed = pool.map(_render, [(s, W, H, D, recipe) for s in seeds], chunksize=2)
    return [pair for pairs in per_seed for pair in pairs]


def label_pass(_lib, left, right, p, p_plain, ws_l, ws_p):
    """Features, winners and labels of one stereo pair (device tensors)."""
    import torch
    lo = _lib.sf_sgm_learned(left, right, p, packed=None, features=True, ws=ws_l)
    po = _lib.sf_sgm_full(left, right, p_plain, ws=ws_p)
    H, W = left.shape
    xs = torch.arange(W, device=left.device).view(1, W)
    labels = po["valid"].clone()
    labels[(xs - lo["dint"].to(torch.int32)) < 0] = 255
    return lo["features"], lo["dint"], labels


def make_dataset(_lib, pairs, D, crop=128, crops_per_scene=2, seed=0):
    """Random crops of features and labels from every pair."""
    import torch
    rng = np.random.default_rng(seed)
    H, W = pairs[0][0].shape
    p = _lib.params(D=D)
    ws_l = _lib.learned_workspace(W, H, p, 1, "cuda")
    ws_p = _lib.workspace(W, H, p, "cuda")
    feats, labs = [], []
    for left, right in pairs:
        f, _, lab = label_pass(_lib, torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(),
                               p, p, ws_l, ws_p)
        for _ in range(crops_per_scene):
            y0 = int(rng.integers(0, H - crop + 1))
            x0 = int(rng.integers(0, W - crop + 1))
            feats.append(f[y0:y0 + crop, x0:x0 + crop].clone())
            labs.append(lab[y0:y0 + crop, x0:x0 + crop].clone())
    return torch.stack(feats), torch.stack(labs)


def train(_lib, feats, labels, epochs=12, batch=16, lr=2e-3, w_neg=2.0, seed=0, log=print):
    import torch
    from paper_1801_04720_gb300 import synth
    params = torch.from_numpy(synth.confnet_init(seed, LAYERS)).cuda()
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    n, crop = feats.shape[0], feats.shape[1]
    ws = _lib.confnet_train_workspace(batch, crop, crop, "cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(seed)
    step = 0
    for ep in range(epochs):
        order = rng.permutation(n)
        tot, cnt = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            idx = torch.from_numpy(order[b0:b0 + batch]).cuda()
            fb, lb = feats.index_select(0, idx).contiguous(), labels.index_select(0, idx).contiguous()
            step += 1
            lr_t = lr * 0.5 * (1 + np.cos(np.pi * min(1.0, step / (epochs * (n // batch)))))
            _lib.confnet_train_step(params, m, v, fb, lb, _lib.hparams(lr=lr_t, w_neg=w_neg, step=step),
                                    ws=ws, loss=loss)
            tot += float(loss.item())
            cnt += 1
        log(f"epoch {ep + 1}/{epochs}: mean loss {tot / max(cnt, 1):.4f}")
    return params


def decisions(_lib, packed, pairs, D):
    """Per pair: probability, winners and plain validity (device tensors)."""
    import torch
    H, W = pairs[0][0].shape
    p = _lib.params(D=D)
    ws_l = _lib.learned_workspace(W, H, p, 1, "cuda")
    ws_p = _lib.workspace(W, H, p, "cuda")
    out = []
    for left, right in pairs:
        l, r = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
        lo = _lib.sf_sgm_learned(l, r, p, packed=packed, threshold=0.5, ws=ws_l)
        po = _lib.sf_sgm_full(l, r, p, ws=ws_p)
        out.append((lo["prob"], lo["dint"], po["valid"]))
    return out


def rates(dec, threshold):
    """False-accept rate (accepted by the learned rule, removed by the plain
    check) over the plain-removed pixels the network decides (x - d* >= 0),
    false-reject rate over the plain-kept pixels, and the accepted fraction."""
    import torch
    fa = neg = fr = pos = acc = tot = 0
    for prob, dint, valid in dec:
        W = prob.shape[1]
        xs = torch.arange(W, device=prob.device).view(1, W)
        decided = (xs - dint.to(torch.int32)) >= 0
        accept = decided & (prob >= threshold)
        plain = valid == 1
        fa += int((accept & ~plain & decided).sum())
        neg += int((~plain & decided).sum())
        fr += int((~accept & plain).sum())
        pos += int(plain.sum())
        acc += int(accept.sum())
        tot += prob.numel()
    return {"false_accept": fa / max(neg, 1), "false_reject": fr / max(pos, 1),
            "accepted": acc / max(tot, 1), "plain_kept": pos / max(tot, 1)}


def accuracy(disps, gts, tau=3.0):
    """Density (fraction of pixels with a disparity, i.e. not NaN) and the
    fraction of those more than `tau` px from the ground truth, over pairs of
    (disparity map, ground-truth disparity) device tensors."""
    import torch
    kept = bad = tot = 0
    for disp, gt in zip(disps, gts):
        m = ~torch.isnan(disp)
        kept += int(m.sum())
        bad += int(((disp - gt).abs() > tau)[m].sum())
        tot += disp.numel()
    return {"density": kept / max(tot, 1), f"bad_{tau:g}px": bad / max(kept, 1)}


def calibrate(dec, target=0.01):
    """Smallest threshold on a grid whose false-accept rate is <= target."""
    for t in np.linspace(0.05, 0.995, 190):
        if rates(dec, float(t))["false_accept"] <= target:
            return float(t)
    return 0.995


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--scenes", type=int, default=len(TRAIN_SEEDS))
    ap.add_argument("--auto-scenes", type=int, default=len(AUTO_TRAIN_SEEDS))
    ap.add_argument("--eval", type=int, default=len(EVAL_SEEDS))
    ap.add_argument("--auto-eval", type=int, default=len(AUTO_EVAL_SEEDS))
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--W", type=int, default=1242)
    ap.add_argument("--H", type=int, default=375)
    ap.add_argument("--D", type=int, default=128)
    ap.add_argument("--target", type=float, default=0.008,
                    help="false-accept rate the threshold is calibrated to, on the held-out "
                         "scenes of each recipe")
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    args = ap.parse_args(argv)
    import torch
    from paper_1801_04720_gb300 import _lib, build
    t0 = time.time()
    size = (args.W, args.H, args.D)
    train_pairs = (render_pairs(list(TRAIN_SEEDS)[:args.scenes], *size)
                   + render_pairs(list(AUTO_TRAIN_SEEDS)[:args.auto_scenes], *size, recipe="automotive"))
    calib = {"planes": render_pairs(list(CALIB_SEEDS), *size),
             "automotive": render_pairs(list(AUTO_CALIB_SEEDS), *size, recipe="automotive")}
    evals = {"planes": (list(EVAL_SEEDS)[:args.eval], render_pairs(list(EVAL_SEEDS)[:args.eval], *size)),
             "automotive": (list(AUTO_EVAL_SEEDS)[:args.auto_eval],
                            render_pairs(list(AUTO_EVAL_SEEDS)[:args.auto_eval], *size, recipe="automotive"))}
    print(f"rendered {len(train_pairs)} training pairs in {time.time() - t0:.1f} s")
    build.build()
    _lib.load()
    t1 = time.time()
    feats, labels = make_dataset(_lib, train_pairs, args.D)
    print(f"dataset {tuple(feats.shape)} in {time.time() - t1:.1f} s")
    t2 = time.time()
    params = train(_lib, feats, labels, epochs=args.epochs)
    torch.cuda.synchronize()
    print(f"trained in {time.time() - t2:.1f} s")
    packed = _lib.confnet_pack(params)
    # the threshold keeps the false-accept rate within the target on each recipe
    threshold = max(calibrate(decisions(_lib, packed, pairs, args.D), target=args.target)
                    for pairs in calib.values())
    ev = {name: {"seeds": [seeds[0], seeds[-1]], "pairs": len(pairs),
                 **rates(decisions(_lib, packed, pairs, args.D), threshold)}
          for name, (seeds, pairs) in evals.items() if seeds}
    meta = {"threshold": threshold, "calibration_target": args.target, "eval": ev,
            "train_pairs": len(train_pairs),
            "calib_seeds": {"planes": [CALIB_SEEDS.start, CALIB_SEEDS.stop - 1],
                            "automotive": [AUTO_CALIB_SEEDS.start, AUTO_CALIB_SEEDS.stop - 1]},
            "size": list(size), "epochs": args.epochs}
    print(json.dumps(meta))
    np.savez(args.out, params=params.cpu().numpy(), meta=json.dumps(meta))
    return meta


def load(path=DEFAULT_WEIGHTS):
    """(fp32 parameters as numpy, metadata dict) of a trained network."""
    z = np.load(path)
    return z["params"].astype(np.float32), json.loads(str(z["meta"]))


if __name__ == "__main__":
    main()
