"""Throughput benchmark of the scene-flow hot path (SGM at t and t+1 with the
left-right check, then the combination) on 1242x375 stereo quadruples, D=128.

One step = one whole frame: sf_scene_flow on one synthetic quadruple resident
in HBM.  Prints ONE JSON line (rank 0).  See --help for the arms."""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "scene-flow frames/s @1242x375 D=128 (learned vs plain L-R); % of HBM roofline"
W_IMG, H_IMG, D_MAX = 1242, 375, 128
WORKLOAD = "automotive 1242x375 D=128 quadruple, plain SGM (8 paths, census 9x7, P1=7, P2=86, L-R tol 1) + combination"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in sweep shape instead of the tuned one")
    ap.add_argument("--batch", type=int, default=64,
                    help="quadruples in the uneven-batch measurement (0 = skip)")
    ap.add_argument("--learned-eval", type=int, default=None,
                    help="held-out scenes for the learned path's false-accept rate "
                         "(0 = timing only, -1 = skip the learned path; default 200, "
                         "-1 under --profile)")
    ap.add_argument("--stream", type=int, default=2,
                    help="frames of the 2048x1024, D=256 stream recipe to time (0 = skip)")
    ap.add_argument("--shape", default=None,
                    help="sweep schedule for the frame's disparity class instead of the "
                         "autotuner: DCxHALO (two launches, e.g. 16x16) or DCxHALOoORDER "
                         "(e.g. 16x8o1: both scan orders in one launch), as in profiling runs")
    ap.add_argument("--profile", action="store_true",
                    help="short run for ncu: no clock-sampling load phase, no e2e, no CPU baseline")
    args = ap.parse_args()
    if args.profile:
        args.no_e2e = True
        args.no_cpu_baseline = True
        args.batch = 0
        args.no_autotune = True
        args.stream = 0
    if args.learned_eval is None:
        args.learned_eval = -1 if args.profile else 200
    return args


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def max_over_ranks(x, world, device):
    """The largest of every rank's x (all ranks get it); x itself at N = 1."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_rate(ms_max, world, units_per_step=1):
    """Whole-job throughput of `world` replicas that each process
    units_per_step units in ms_max milliseconds (the slowest rank's time)."""
    return world * units_per_step * 1000.0 / ms_max


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.t0 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [v.strip() for v in line.split(",")]))

    def mark(self):
        self.t0 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for t, r in self.rows if self.t0 is None or t >= self.t0 - 0.1]
        if not rows:
            rows = [r for _, r in self.rows[-3:]]
        sm = [float(r[1]) for r in rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def bytes_model(stage, N, D, passes=4, order=1):
    """Algorithmic HBM bytes per launch of the dominant stage.

    sgm_sweep: the eight paths run in opposite scan orders, so the partial sum
    of the paths of one order must exist for every (p, d) when the opposite
    order reaches p: per SGM pass it is written once and read once (uint16,
    2*N*D bytes each way).  One launch covers the four passes of a frame.
    With both scan orders in one launch (orders 1 and 2) that launch does the
    write and the read -> 4 * 4*N*D bytes; with one launch per order (order 0)
    each does one of them -> 4 * 2*N*D bytes.  With order 2 the launch also
    runs the horizontal paths: per pass the uint8 cost read once and both
    uint8 path volumes written -> + 4 * 3*N*Dp bytes.
    aggregate (the horizontal paths' own launch): the same 3*N*Dp per pass."""
    Dp = (D + 15) // 16 * 16
    if stage == "sgm_sweep":
        return passes * (4 if order >= 1 else 2) * N * D + (passes * 3 * N * Dp if order == 2 else 0)
    return passes * 3 * N * Dp


def densify_bytes_model(N):
    """Algorithmic HBM bytes of one sf_densify_sceneflow call on a frame:
    per map (d0, d1) the row pass reads the sparse value twice and writes it
    twice (the parked index, then the value: 16 N); then the dense
    back-projection reads the flow and s4 (24 N) and writes s4, motion, point
    and validity (41 N).  The column pass touches only rows with nothing
    kept (none on these frames)."""
    return 2 * 16 * N + 24 * N + 41 * N


def run_densify(_lib, torch, out, flow, cam, guide, stream, flush, N):
    """Time of the densification call on the frame's sparse output, both
    modes (L2 flushed between calls)."""
    H, W = out["s4"].shape[:2]
    dev = out["s4"].device
    dn = {"s4": torch.empty((H, W, 4), dtype=torch.float32, device=dev),
          "motion": torch.empty((H, W, 3), dtype=torch.float32, device=dev),
          "point": torch.empty((H, W, 3), dtype=torch.float32, device=dev),
          "valid": torch.empty((H, W), dtype=torch.uint8, device=dev)}
    res = {"call": "sf_densify_sceneflow on the frame's sparse s4 (fill_rows, fill_cols, backproject kernels)"}
    hbm_peak = peaks()[0]
    for mode, tag in ((0, "background"), (1, "edge_aware")):
        for _ in range(3):
            _lib.sf_densify_sceneflow(out["s4"], flow, cam, guide=guide, mode=mode, out=dn, stream=stream)
        ms = []
        for k in range(20):
            flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _lib.sf_densify_sceneflow(out["s4"], flow, cam, guide=guide, mode=mode, out=dn, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = statistics.mean(ms)
        b = densify_bytes_model(N) + (N if mode == 1 else 0)
        res[tag] = {"ms_per_call": round(t, 4), "model_bytes": b,
                    "achieved_gbs": round(b / (t * 1e-3) / 1e9, 1),
                    "frac": round(b / (t * 1e-3) / 1e9 / hbm_peak, 4)}
    res["model"] = "densify_bytes_model: 97 N (+ N guide reads in the edge-aware mode)"
    return res


def stage_bytes_model(stage, N, D, passes=4, order=1):
    """Algorithmic HBM bytes per frame of each stage of the plain path as the
    kernels are built (stored cost and horizontal volumes included):
    census: four images in, four uint64 strings out (36 N);
    cost: the strings in, both references' uint8 volumes of both pairs out
      (32 N + 4 N Dp);
    aggregate (horizontal paths): per pass the cost in and both uint8 path
      volumes out (3 N Dp);
    sgm_sweep: the partial sums of one scan order written and read, uint16
      (4 N D per pass; the stored volumes it also reads are not counted),
      plus the horizontal paths' 3 N Dp per pass when the launch runs them
      (order 2);
    combine (both checks and the combination): winners and subpixel maps of
      both pairs and the flow in (24 N), both disparity maps, s4, motion,
      point and validity out (49 N)."""
    Dp = (D + 15) // 16 * 16
    return {"census": 36 * N, "cost": 32 * N + passes * N * Dp,
            "aggregate": passes * 3 * N * Dp,
            "sgm_sweep": passes * 4 * N * D + (passes * 3 * N * Dp if order == 2 else 0),
            "combine": 73 * N}.get(stage)


def frame_bytes_model(N, D):
    """Algorithmic HBM bytes of one plain scene-flow frame (4 SGM passes and
    the combination) for a design that stores nothing but the partial sum of
    one scan order: per pass that uint16 sum is written once and read once
    (4 N D), 16 N D over the passes; plus the four images in (4 N), their
    census strings written and read (64 N), the integer winners of the four
    passes written and read by the checks (16 N), both disparity maps
    written and read (16 N), the flow in (8 N) and the outputs out (s4,
    motion, point, valid: 41 N)."""
    return 16 * N * D + 149 * N


def measured_traffic(stage, shape=None):
    """DRAM bytes per launch of `stage` from the committed ncu captures, or
    None when there is none for the sweep shape ("DCxHALO") timed, or the
    kernel sources changed since they were taken."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(prof)).get(stage)
        h = hashlib.sha256()
        for src in rec["sources"]:
            h.update(open(os.path.join(ROOT, src), "rb").read())
        if h.hexdigest() != rec["sources_sha256"]:
            return None
        if "by_shape" in rec:
            return rec["by_shape"][shape]["bytes_per_launch"] if shape in rec["by_shape"] else None
        if rec.get("shape", "any") != "any" and rec.get("shape") != shape:
            return None
        return rec["bytes_per_launch"]
    except (OSError, ValueError, KeyError, TypeError, AttributeError):
        return None


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_1801_04720_gb300 import _lib, build, synth

    torch.cuda.set_device(local)
    build.build()
    _lib.load()
    dev = torch.device("cuda", local)
    tuned = None
    if args.shape:
        # DCxHALO (two launches) or DCxHALOoORDER
        spec = args.shape.lower()
        order = int(spec.split("o")[1]) if "o" in spec else 0
        dc, halo = (int(v) for v in spec.split("o")[0].split("x"))
        _lib.sf_set_sweep_schedule(65, 128, dc, halo, order)
        tuned = {"classes": [{"lo": 65, "hi": 128, "dc": dc, "halo": halo, "order": order, "forced": True}]}
    elif not args.no_autotune:
        from paper_1801_04720_gb300 import autotune
        # every class of disparity counts the batch uses (64, 128, 192); the
        # learned calls' own table for the frame (128) and the stream (256)
        tuned = autotune.load_or_tune(W=W_IMG, H=H_IMG, classes=[(33, 64), (65, 128), (129, 256)],
                                      learned_classes=[(65, 128), (129, 256)])
    q = synth.automotive(seed=args.seed + rank)
    H, W = q.shape
    N = W * H
    p = _lib.params(D=D_MAX)
    cam = _lib.camera(q.camera.f, q.camera.B, q.camera.cx, q.camera.cy)
    imgs = [torch.from_numpy(im).to(dev) for im in q.images()]
    flow = torch.from_numpy(q.flow).to(dev)
    ws = _lib.workspace(W, H, p, dev)
    out = _lib.alloc_scene_flow_outputs(W, H, dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2
    if not getattr(args, "fused", True):
        _lib.sf_set_fused(False)

    def step():
        _lib.sf_scene_flow(imgs, flow, p, cam, ws=ws, out=out, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # keep the GPU loaded for >= ~1.5 s before and during the timed region so
    # the clock samples describe the timed work
    clocks = ClockSampler(local)
    if not args.profile:
        clocks.start()
        t_end = time.time() + 1.5
        while time.time() < t_end:
            step()
            torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.mark()
    launches0 = _lib.kernel_launches()
    # timed steps: nothing but the frame between the two events
    for k in range(args.steps):
        flush.fill_(k & 0xFF)            # L2 flush between timed steps (untimed)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    launches = _lib.kernel_launches() - launches0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = max_over_ranks(statistics.mean(step_ms), world, dev)
    # the same steps once more with the per-stage event pairs (stage times and
    # the dominant kernel's launch duration; timestamped events between the
    # launches can cost the frame some overlap, so not part of the timed run)
    tracer = _lib.StageTracer(n_records=64 * args.steps)
    with tracer:
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            step()
    torch.cuda.synchronize()
    stages = tracer.durations()
    stage_tot = {k: sum(v) for k, v in stages.items()}
    dominant = max(stage_tot, key=stage_tot.get)
    dom_ms = statistics.mean(stages[dominant])
    hbm_peak, peak_kind = peaks()
    cls = [c for c in (tuned or {}).get("classes", []) if c["lo"] <= D_MAX <= c["hi"]]
    if cls:
        order = cls[0].get("order", 0)
        shape_now = f'{cls[0]["dc"]}x{cls[0]["halo"]}o{order}'
    else:
        order = 1
        shape_now = "16x8o1"   # built-in rule for D = 128
    algo_bytes = bytes_model(dominant, N, D_MAX, order=order)
    achieved = algo_bytes / (dom_ms * 1e-3) / 1e9
    traffic = measured_traffic(dominant, shape_now)

    e2e = None
    if not args.no_e2e:
        ws_h = torch.empty(_lib.sf_scene_flow_host_workspace_size(W, H, p), dtype=torch.uint8,
                           device=dev)
        h_imgs = [torch.from_numpy(im).pin_memory() for im in q.images()]
        h_flow = torch.from_numpy(q.flow).pin_memory()
        h_out = {"s4": torch.empty((H, W, 4)).pin_memory(),
                 "motion": torch.empty((H, W, 3)).pin_memory(),
                 "point": torch.empty((H, W, 3)).pin_memory(),
                 "valid": torch.empty((H, W), dtype=torch.uint8).pin_memory()}
        for _ in range(3):
            _lib.sf_scene_flow_host(h_imgs, h_flow, p, cam, ws_h, h_out, stream=stream)
        # latency of one synchronous call (L2 flushed before each)
        lat = []
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _lib.sf_scene_flow_host(h_imgs, h_flow, p, cam, ws_h, h_out, stream=stream)
            lat.append((time.perf_counter() - t0) * 1e3)
        del ws_h
        # throughput through the frame pipeline: every step copies its inputs
        # in from pinned host memory and its outputs back, overlapped with the
        # neighbouring frames' computation; the host waits for a frame's
        # outputs before it hands their buffers to a later frame
        depth = 2
        h_outs = [h_out] + [{k: torch.empty_like(v).pin_memory() for k, v in h_out.items()}
                            for _ in range(depth - 1)]
        with _lib.Pipeline(W, H, p, cam, depth=depth) as pl:
            for k in range(2 * depth):
                if k >= depth:
                    pl.wait(k - depth)
                pl.submit(h_imgs, h_flow, h_outs[k % depth])
            pl.wait(2 * depth - 1)
            if world > 1:
                torch.distributed.barrier()
            t0 = time.perf_counter()
            for k in range(args.steps):
                if k >= depth:
                    pl.wait(k - depth + 2 * depth)
                pl.submit(h_imgs, h_flow, h_outs[k % depth])
            pl.wait(2 * depth + args.steps - 1)
            e_total = (time.perf_counter() - t0) * 1e3
        e_mean = max_over_ranks(e_total / args.steps, world, dev)
        e2e = {"value": round(replica_rate(e_mean, world), 2), "unit": "frames/s",
               "h2d_bytes_per_step": 4 * N + 8 * N, "d2h_bytes_per_step": 16 * N + 12 * N + 12 * N + N,
               "ms_per_step": round(e_mean, 4),
               "api": f"sf_pipeline_submit / sf_pipeline_wait, {depth} slots, pinned host buffers",
               "l2": "not flushed in the pipelined run: each step's inputs arrive by copy from host "
                     "memory and a frame's 0.9 GB working set exceeds the L2",
               "latency_ms_sf_scene_flow_host": round(max_over_ranks(statistics.mean(lat), world, dev), 4)}

    result = {
        "metric": METRIC, "value": round(replica_rate(ms, world), 2), "unit": "frames/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8/u16 integer SGM, f32 subpixel + scene flow",
        "data": "synthetic (seeded automotive-shaped scenes; KITTI is not available)",
        "config": {"workload": WORKLOAD, "W": W, "H": H, "D": D_MAX, "frames_per_step": 1,
                   "path": "plain L-R", "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MB write, untimed)"},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": round(achieved, 1),
                     "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                     "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": algo_bytes,
                     "avg_launch_ms": round(dom_ms, 5)},
        "frame_hbm": {"model_bytes_per_frame": frame_bytes_model(N, D_MAX),
                      "achieved_gbs": round(frame_bytes_model(N, D_MAX) / (ms * 1e-3) / 1e9, 1),
                      "frac": round(frame_bytes_model(N, D_MAX) / (ms * 1e-3) / 1e9 / hbm_peak, 4),
                      "model": "frame_bytes_model: 16 N D + 149 N"},
        "stages_ms_per_step": {k: round(v / args.steps, 5) for k, v in stage_tot.items()},
        "stages_hbm": {k: {"model_bytes": stage_bytes_model(k, N, D_MAX, order=order),
                           "frac": round(stage_bytes_model(k, N, D_MAX, order=order) / (v / args.steps * 1e-3)
                                         / 1e9 / hbm_peak, 4)}
                       for k, v in stage_tot.items() if stage_bytes_model(k, N, D_MAX, order=order)},
        "clocks": clk, "e2e": e2e, "gpu_launches": int(launches),
        "sweep_shape": tuned["classes"] if tuned else "built-in",
        "learned_sweep_shape": (tuned.get("learned") or "built-in") if tuned else "built-in",
    }
    # KITTI-style accuracy of this frame's output against the scene's ground truth
    from paper_1801_04720_gb300 import evaluate
    step()
    torch.cuda.synchronize()
    s4_h, valid_h = out["s4"].cpu(), out["valid"].cpu()
    result["accuracy_vs_ground_truth"] = {
        "rule": "outlier: error > 3 px and > 5 % of the true value; rates over the kept pixels",
        "plain": {k: round(v, 5) for k, v in evaluate.scene_flow_accuracy(
            s4_h, valid_h, q.gt_disp0, q.gt_disp1, q.gt_flow).items()},
        "dense": "d0 and d1 filled by the densification kernels (sf_densify_sceneflow): the "
                 "background fill (the benchmark's reading) or the edge-aware fill guided by the left "
                 "image, (u, v) from the input flow, back-projected at every pixel"}
    for mode, tag in ((0, "plain_dense"), (1, "plain_dense_edge_aware")):
        dn = _lib.sf_densify_sceneflow(out["s4"], flow, cam, guide=imgs[0], mode=mode, stream=stream)
        torch.cuda.synchronize()
        result["accuracy_vs_ground_truth"][tag] = {k: round(v, 5) for k, v in evaluate.scene_flow_accuracy(
            dn["s4"].cpu(), dn["valid"].cpu(), q.gt_disp0, q.gt_disp1, q.gt_flow).items()}
    result["densify"] = run_densify(_lib, torch, out, flow, cam, imgs[0], stream, flush, N)
    if args.batch > 0:
        result["batch"] = run_batch(args, dev, _lib, synth, torch)
    if args.learned_eval >= 0:
        result["learned"] = run_learned(args, dev, _lib, torch, q, imgs, flow, p, cam, flush,
                                        result["value"])
    if args.stream > 0:
        result["stream"] = run_stream(args, dev, _lib, torch, flush)
    return result, q


def run_batch(args, dev, _lib, synth, torch):
    """Uneven batch: quadruples with sizes drawn from {320x240, 640x480,
    1024x320, 1242x375} and D from {64, 128, 192} (fronto-parallel plane
    recipe), all in one sf_batch_run per step, replayed as a CUDA graph."""
    quads = [synth.batch_recipe(seed=k) for k in range(args.batch)]
    scenes, outs = [], []
    for q in quads:
        scenes.append({"left_t": torch.from_numpy(q.left_t).to(dev),
                       "right_t": torch.from_numpy(q.right_t).to(dev),
                       "left_t1": torch.from_numpy(q.left_t1).to(dev),
                       "right_t1": torch.from_numpy(q.right_t1).to(dev),
                       "flow": torch.from_numpy(q.flow).to(dev), "D": q.D,
                       "cam": _lib.camera(q.camera.f, q.camera.B, q.camera.cx, q.camera.cy)})
        outs.append(_lib.alloc_scene_flow_outputs(q.shape[1], q.shape[0], dev))
    items = _lib.make_batch(scenes, outs)
    p = _lib.params()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    steps = max(3, min(args.steps, 10))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    def measure(limit):
        """quadruples/s and workspace bytes with the batch in waves of at most
        `limit` bytes of buffers (0: one wave)."""
        _lib.sf_set_batch_wave_limit(limit)
        ws = torch.empty(_lib.sf_batch_workspace_size(items, p), dtype=torch.uint8, device=dev)
        for _ in range(max(2, args.warmup)):
            _lib.sf_batch_run(items, p, ws, graph=True, stream=stream)
        torch.cuda.synchronize()
        ms = []
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _lib.sf_batch_run(items, p, ws, graph=True, stream=stream)
                e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        _lib.sf_batch_release_graphs()
        n = ws.numel()
        del ws
        torch.cuda.empty_cache()
        return max_over_ranks(statistics.mean(ms), world, dev), n

    mean, ws_all = measure(0)
    wave_limit = 8 << 30
    mean_w, ws_w = measure(wave_limit)
    _lib.sf_set_batch_wave_limit(0)
    pixels = sum(q.shape[0] * q.shape[1] for q in quads)
    return {"metric": "scene-flow quadruples/s, uneven batch",
            "value": round(replica_rate(mean, world, len(quads)), 2),
            "unit": "quadruples/s", "items": len(quads), "ms_per_step": round(mean, 3),
            "megapixels_per_step": round(pixels / 1e6, 3),
            "workspace_gb": round(ws_all / 1e9, 2), "graph": True,
            "waves": {"limit_gb": round(wave_limit / 1e9, 2), "workspace_gb": round(ws_w / 1e9, 2),
                      "value": round(replica_rate(mean_w, world, len(quads)), 2), "unit": "quadruples/s",
                      "ms_per_step": round(mean_w, 3)},
            "sizes": sorted({f"{q.shape[1]}x{q.shape[0]}/D{q.D}" for q in quads})}


def run_learned(args, dev, _lib, torch, q, imgs, flow, p, cam, flush, plain_fps):
    """The same frame with learned confidence in place of both left-right
    checks (two SGM passes + features + network + combination), and its
    false-accept / false-reject rates against the plain check: on this frame
    and on the held-out plane-recipe scenes at 1242x375, D=128."""
    from paper_1801_04720_gb300 import synth, train_confnet
    theta, meta = train_confnet.load()
    params_t = torch.from_numpy(theta).to(dev)
    packed = _lib.confnet_pack(params_t)
    thr = float(meta["threshold"])
    H, W = q.shape
    ws = _lib.learned_workspace(W, H, p, 2, dev)
    out = _lib.alloc_scene_flow_outputs(W, H, dev)
    stream = torch.cuda.current_stream()

    def step():
        _lib.sf_scene_flow_learned(imgs, flow, p, cam, packed, thr, ws=ws, out=out, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = _lib.kernel_launches()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    launches = _lib.kernel_launches() - launches0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    ms = max_over_ranks(statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends)), world, dev)
    tracer = _lib.StageTracer(n_records=64 * args.steps)
    with tracer:
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            step()
    torch.cuda.synchronize()
    stages = {k: round(sum(v) / args.steps, 5) for k, v in tracer.durations().items()}
    # two frames per launch (their four left passes fill the GPU like the four
    # passes of one plain frame): the second frame is the next seed's scene
    q2 = synth.automotive(seed=args.seed + 1000)
    imgs2 = [torch.from_numpy(im).to(dev) for im in q2.images()]
    flow2 = torch.from_numpy(q2.flow).to(dev)
    ws2 = _lib.learned_workspace(W, H, p, 4, dev)
    outs2 = [_lib.alloc_scene_flow_outputs(W, H, dev) for _ in range(2)]
    scenes2 = [(imgs, flow), (imgs2, flow2)]

    def step2():
        _lib.sf_scene_flow_learned_frames(scenes2, p, cam, packed, thr, ws=ws2, outs=outs2, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step2()
    torch.cuda.synchronize()
    ms2 = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step2()
        e1.record(stream)
        torch.cuda.synchronize()
        ms2.append(e0.elapsed_time(e1))
    ms2 = max_over_ranks(statistics.mean(ms2), world, dev)
    # accuracy against the plain check on this frame (pair at t)
    plain = _lib.sf_sgm_full(imgs[0], imgs[1], p)
    lo = _lib.sf_sgm_learned(imgs[0], imgs[1], p, packed=packed, threshold=thr)
    frame_rates = train_confnet.rates([(lo["prob"], lo["dint"], plain["valid"])], thr)
    gt = [torch.from_numpy(q.gt_disp0).to(dev)]
    frame_gt = {"plain_check": train_confnet.accuracy([plain["disp"]], gt),
                "learned": train_confnet.accuracy([lo["disp"]], gt)}
    from paper_1801_04720_gb300 import evaluate
    step()
    torch.cuda.synchronize()
    sf_acc = evaluate.scene_flow_accuracy(out["s4"].cpu(), out["valid"].cpu(), q.gt_disp0, q.gt_disp1,
                                          q.gt_flow)
    res = {"metric": "scene-flow frames/s, learned confidence in place of the L-R check",
           "value": round(replica_rate(ms, world), 2), "unit": "frames/s", "ms_per_step": round(ms, 4),
           "vs_plain": round(replica_rate(ms, world) / plain_fps, 3), "threshold": thr,
           "two_frames_per_launch": {"value": round(replica_rate(ms2, world, 2), 2), "unit": "frames/s",
                                     "ms_per_step": round(ms2, 4),
                                     "vs_plain": round(replica_rate(ms2, world, 2) / plain_fps, 3)},
           "gpu_launches": int(launches), "stages_ms_per_step": stages,
           "automotive_frame": {k: round(v, 5) for k, v in frame_rates.items()},
           "automotive_frame_vs_ground_truth": {k: {kk: round(vv, 5) for kk, vv in v.items()}
                                                for k, v in frame_gt.items()},
           "scene_flow_accuracy_vs_ground_truth": {k: round(v, 5) for k, v in sf_acc.items()}}
    n_eval = min(args.learned_eval, len(train_confnet.EVAL_SEEDS))
    if n_eval > 0:
        # held-out scenes of both training recipes (never trained or calibrated on)
        res["eval"] = {}
        for name, all_seeds, n, recipe in (
                ("planes", train_confnet.EVAL_SEEDS, n_eval,
                 "fronto-parallel plane recipe at 1242x375, D=128, pair at t"),
                ("automotive", train_confnet.AUTO_EVAL_SEEDS, min(max(n_eval // 4, 1), len(train_confnet.AUTO_EVAL_SEEDS)),
                 "automotive recipe at 1242x375, D=128, pairs at t and t+1")):
            seeds = list(all_seeds)[:n]
            pairs = train_confnet.render_pairs(seeds, W, H, D_MAX, recipe=name)
            ev = train_confnet.rates(train_confnet.decisions(_lib, packed, pairs, D_MAX), thr)
            res["eval"][name] = {"scenes": n, "pairs": len(pairs), "seeds": [seeds[0], seeds[-1]],
                                 "recipe": recipe, **{k: round(v, 5) for k, v in ev.items()}}
    return res


STREAM_K = 32            # consecutive frames of the large-stream sequence
STREAM_SEED = 5


def _stream_frames(frames):
    """Worker: frames of the large-stream sequence (the scene depends on the
    seed alone, so any subset renders on its own)."""
    from paper_1801_04720_gb300 import synth
    sq = synth.sequence(STREAM_K, seed=STREAM_SEED, W=2048, H=1024, D=256, n_segments=40, frames=frames)
    last = STREAM_K - 1
    return [(k, sq.lefts[k], sq.rights[k], sq.flows[k] if k < last else None, sq.gt_disp[k],
             sq.gt_flow[k] if k < last else None, sq.gt_next_disp[k] if k < last else None)
            for k in frames], sq.camera


def _oracle_sgm_pass(task):
    """Worker: one SGM pass of the oracle (census, cost, eight paths, selection)."""
    from oracle import oracle
    ref, oth, is_right, D = task
    return oracle.sgm_pass(oracle.census(ref), oracle.census(oth), D, 7, 86, is_right, 62,
                           subpixel=not is_right)


def _mem_available_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


def sequence_bytes_model(N, D):
    """Algorithmic HBM bytes per frame of a sequence in which every stereo
    frame's SGM runs once: its two passes' partial sums written and read
    (2 x 4 N D), its two images in (2 N), census strings written and read
    (2 x 8 N x 2), the winners of both passes written and read (8 N), its
    disparity map written once and read by two combinations (12 N), one flow
    in (8 N) and one step's s4 and validity out (17 N)."""
    return 8 * N * D + 2 * N + 32 * N + 8 * N + 12 * N + 8 * N + 17 * N


def run_stream(args, dev, _lib, torch, flush):
    """The large-stream configuration: 32 consecutive 2048x1024 stereo frames
    (D = 256) of one driving scene with 40 moving segments, through the
    sequence call (every frame's SGM once, a scene-flow step per consecutive
    pair) with the plain left-right check and with learned confidence (four
    left passes per launch), the plain check judging the learned one, and the
    oracle on frames 0 and 1 (host workers, beside the GPU timing)."""
    import multiprocessing as mp
    from oracle import oracle
    from paper_1801_04720_gb300 import evaluate, train_confnet
    oracle.build()
    K = STREAM_K
    D = 256
    cores = max(1, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    t_render = time.perf_counter()
    with ctx.Pool(min(cores, 16)) as pool:
        parts = pool.map(_stream_frames, [list(range(i, K, min(cores, 16))) for i in range(min(cores, 16))])
    t_render = time.perf_counter() - t_render
    cam_h = parts[0][1]
    fr = {}
    for lst, _ in parts:
        for k, l_, r_, f_, gd, gf, gn in lst:
            fr[k] = (l_, r_, f_, gd, gf, gn)
    H, W = fr[0][0].shape
    N = W * H
    # the oracle on frames 0 and 1 (four SGM passes) in spawned workers while
    # the GPU is timed; each pass holds about 5 GB of host memory
    n_or = int(min(4, max(0, _mem_available_gb() // 6)))
    or_pool = ctx.Pool(n_or) if n_or else None
    or_async = None
    if or_pool is not None:
        tasks = []
        for k in (0, 1):
            l_, r_ = fr[k][0], fr[k][1]
            tasks += [(l_, r_, False, D), (r_, l_, True, D)]
        or_async = or_pool.map_async(_oracle_sgm_pass, tasks)
    p = _lib.params(D=D)
    cam = _lib.camera(cam_h.f, cam_h.B, cam_h.cx, cam_h.cy)
    L = [torch.from_numpy(fr[k][0]).to(dev) for k in range(K)]
    R = [torch.from_numpy(fr[k][1]).to(dev) for k in range(K)]
    F = [torch.from_numpy(fr[k][2]).to(dev) for k in range(K - 1)]
    stream = torch.cuda.current_stream()
    theta, meta = train_confnet.load()
    packed = _lib.confnet_pack(torch.from_numpy(theta).to(dev))
    thr = float(meta["threshold"])
    ws_p = torch.empty(_lib.load().sf_sequence_workspace_size(W, H, __import__("ctypes").byref(p), K, 0),
                       dtype=torch.uint8, device=dev)
    ws_l = torch.empty(_lib.load().sf_sequence_workspace_size(W, H, __import__("ctypes").byref(p), K, 1),
                       dtype=torch.uint8, device=dev)
    steps = max(3, min(args.steps, 5))

    def timed(fn):
        out = fn()
        torch.cuda.synchronize()
        ms = []
        for k in range(steps):
            flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.mean(ms), out

    out_p = _lib.alloc_sequence_outputs(K, W, H, dev)
    out_l = _lib.alloc_sequence_outputs(K, W, H, dev)
    ms_plain, _ = timed(lambda: _lib.sf_sequence_sceneflow(L, R, F, p, cam, ws=ws_p, out=out_p, stream=stream))
    ms_learn, _ = timed(lambda: _lib.sf_sequence_sceneflow(L, R, F, p, cam, packed=packed, threshold=thr,
                                                           ws=ws_l, out=out_l, stream=stream))
    # the plain check judges the learned rule on every frame
    dec, dp, dl, gts = [], [], [], []
    ws1 = _lib.learned_workspace(W, H, p, 1, dev)
    wsf = _lib.workspace(W, H, p, dev)
    for k in range(K):
        plain = _lib.sf_sgm_full(L[k], R[k], p, ws=wsf)
        lo = _lib.sf_sgm_learned(L[k], R[k], p, packed=packed, threshold=thr, ws=ws1, features=False)
        dec.append((lo["prob"], lo["dint"], plain["valid"]))
        dp.append(out_p["disp"][k])
        dl.append(out_l["disp"][k])
        gts.append(torch.from_numpy(fr[k][3]).to(dev))
    rates = train_confnet.rates(dec, thr)
    vs_gt = {"plain_check": train_confnet.accuracy(dp, gts), "learned": train_confnet.accuracy(dl, gts)}
    # scene-flow accuracy of step 0 (frames 0 -> 1), sparse and densified by the kernels
    acc = {}
    for name, o in (("plain", out_p), ("learned", out_l)):
        s4, va = o["s4"][0], o["valid"][0]
        acc[name] = {k: round(v, 5) for k, v in evaluate.scene_flow_accuracy(
            s4.cpu(), va.cpu(), fr[0][3], fr[0][5], fr[0][4]).items()}
        for mode, tag in ((0, "dense_background"), (1, "dense_edge_aware")):
            dn = _lib.sf_densify_sceneflow(s4, F[0], cam, guide=L[0], mode=mode)
            acc[f"{name}_{tag}"] = {k: round(v, 5) for k, v in evaluate.scene_flow_accuracy(
                dn["s4"].cpu(), dn["valid"].cpu(), fr[0][3], fr[0][5], fr[0][4]).items()}
    # the oracle on frames 0 and 1
    parity = {"frames": [0, 1], "unavailable": "not enough host memory for the oracle workers"}
    if or_async is not None:
        t_or = time.perf_counter()
        res = or_async.get()
        or_pool.close()
        or_pool.join()
        disp_o = []
        for f in (0, 1):
            (dL, dLs), (dR, _) = res[2 * f], res[2 * f + 1]
            disp_o.append(oracle.lr_check(dL, dR, dLs, 1)[1])
        s4o, _, _, vo = oracle.combine(disp_o[0], disp_o[1], fr[0][2], cam_h.f, cam_h.B, cam_h.cx, cam_h.cy)
        parity = {"frames": [0, 1], "oracle_workers": n_or, "oracle_wait_s": round(time.perf_counter() - t_or, 1)}
        for f in (0, 1):
            g = out_p["disp"][f].cpu().numpy()
            o = disp_o[f]
            parity[f"frame{f}_validity_mismatches"] = int((np.isnan(g) != np.isnan(o)).sum())
            m = ~np.isnan(o) & ~np.isnan(g)
            parity[f"frame{f}_max_subpixel_err_px"] = float(np.abs(g[m] - o[m]).max()) if m.any() else 0.0
        gv = out_p["valid"][0].cpu().numpy()
        gs = out_p["s4"][0].cpu().numpy()
        parity["step0_validity_mismatches"] = int((gv != vo).sum())
        m = (vo == 1) & (gv == 1)
        rel = np.abs(gs[m].astype(np.float64) - s4o[m]) / np.maximum(np.abs(s4o[m]), 1e-30)
        parity["step0_s4_max_rel_err"] = float(rel.max()) if m.any() else 0.0
    steps_s = (K - 1) * 1000.0 / ms_plain
    bpf = sequence_bytes_model(N, D)
    return {"workload": f"automotive sequence {W}x{H} D={D}, 40 moving segments, {K} consecutive frames "
                        f"(a scene-flow step per consecutive pair)",
            "render_s": round(t_render, 1),
            "plain": {"value": round(steps_s, 2), "unit": "scene-flow frames/s", "ms_per_sequence": round(ms_plain, 3),
                      "stereo_frames_per_s": round(K * 1000.0 / ms_plain, 2),
                      "hbm": {"model_bytes_per_frame": bpf,
                              "achieved_gbs": round(bpf * K / (ms_plain * 1e-3) / 1e9, 1),
                              "peak_gbs": peaks()[0],
                              "frac": round(bpf * K / (ms_plain * 1e-3) / 1e9 / peaks()[0], 4),
                              "model": "sequence_bytes_model: 8 N D + 87 N per stereo frame"}},
            "learned": {"value": round((K - 1) * 1000.0 / ms_learn, 2), "unit": "scene-flow frames/s",
                        "ms_per_sequence": round(ms_learn, 3), "vs_plain": round(ms_plain / ms_learn, 3),
                        "passes_per_launch": 4},
            "learned_vs_plain_check": {k: round(v, 5) for k, v in rates.items()},
            "vs_ground_truth": {k: {kk: round(vv, 5) for kk, vv in v.items()} for k, v in vs_gt.items()},
            "scene_flow_accuracy_step0": acc,
            "oracle_parity": parity}


def cpu_baseline(q):
    """The oracle as it stands on one full frame (single thread), and the
    same frame with the oracle's functions spread over every host core."""
    from oracle import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.scene_flow(q.images(), q.flow, q.camera.f, q.camera.B, q.camera.cx, q.camera.cy,
                      D=D_MAX)
    dt = time.perf_counter() - t0
    out = {"value": round(1.0 / dt, 5), "unit": "frames/s", "cores": 1, "kind": "oracle",
           "sample": "one full 1242x375 D=128 frame (4 SGM passes + combination), 1 thread",
           "seconds": round(dt, 2), "cpu_model": cpu_model()}
    try:
        out["all_cores"] = cpu_baseline_all_cores(q)
    except (OSError, RuntimeError, ValueError) as e:       # e.g. no shared memory on the host
        out["all_cores"] = {"unavailable": str(e)[:200]}
    return out


def cpu_model():
    """The host CPU's model name (x86 'model name', else lscpu's 'Model name')."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        import subprocess
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


# ---- all-cores oracle: the oracle's own functions over independent units ----
# A frame is four SGM passes; each pass is a cost volume and eight path
# aggregations that do not depend on one another.  Phase 1 computes the four
# cost volumes (one task each), phase 2 the 32 (pass, direction) paths, each
# adding its L_r into its pass's sum in shared memory under that pass's lock;
# the selection, checks and combination then run in the parent.
_SHM = {}


def _shm_array(name, shape, dtype):
    from multiprocessing import shared_memory
    if name not in _SHM:
        _SHM[name] = shared_memory.SharedMemory(name=name)
    return np.ndarray(shape, dtype=dtype, buffer=_SHM[name].buf)


def _ac_init(locks):
    global _AC_LOCKS
    _AC_LOCKS = locks


def _ac_cost(task):
    from oracle import oracle
    k, ref, oth, is_right, D, names, shape = task
    C = oracle.cost_volume(oracle.census(ref), oracle.census(oth), D, is_right, 62)
    _shm_array(names["cost"][k], shape, np.uint8)[...] = C
    return k


def _ac_path(task):
    from oracle import oracle
    k, r, names, shape = task
    C = _shm_array(names["cost"][k], shape, np.uint8)
    L = oracle.path_cost(C, 7, 86, r)
    with _AC_LOCKS[k]:
        _shm_array(names["sum"][k], shape, np.int32)[...] += L
    return k


def cpu_baseline_all_cores(q, cores=None, D=None, keep=None):
    """The oracle on one full frame with its independent units spread over
    every host core (spawned workers): frames/s and the cores used.  `keep`
    (a dict) receives the frame's combination outputs."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    from oracle import oracle
    oracle.build()
    cores = cores or os.cpu_count() or 1
    H, W = q.shape
    D = D or D_MAX
    shape = (H, W, D)
    imgs = q.images()
    passes = [(imgs[0], imgs[1], False), (imgs[1], imgs[0], True), (imgs[2], imgs[3], False),
              (imgs[3], imgs[2], True)]
    blocks, names = [], {"cost": [], "sum": []}
    try:
        for k in range(4):
            c = shared_memory.SharedMemory(create=True, size=H * W * D)
            s_ = shared_memory.SharedMemory(create=True, size=H * W * D * 4)
            blocks += [c, s_]
            names["cost"].append(c.name)
            names["sum"].append(s_.name)
        ctx = mp.get_context("spawn")
        locks = [ctx.Lock() for _ in range(4)]
        with ctx.Pool(cores, initializer=_ac_init, initargs=(locks,)) as pool:
            pool.map(abs, range(cores))                   # workers started before the clock
            t0 = time.perf_counter()
            for k in range(4):
                np.ndarray(shape, dtype=np.int32, buffer=blocks[2 * k + 1].buf)[...] = 0
            pool.map(_ac_cost, [(k, passes[k][0], passes[k][1], passes[k][2], D, names, shape)
                                for k in range(4)])
            pool.map(_ac_path, [(k, r, names, shape) for k in range(4) for r in oracle.DIRECTIONS],
                     chunksize=1)
            sel = []
            for k in range(4):
                S = np.ndarray(shape, dtype=np.int32, buffer=blocks[2 * k + 1].buf)
                sel.append(oracle.select(S, subpixel=(k % 2 == 0)))
            disp = []
            for f in range(2):
                (dL, dLs), (dR, _) = sel[2 * f], sel[2 * f + 1]
                disp.append(oracle.lr_check(dL, dR, dLs, 1)[1])
            res = oracle.combine(disp[0], disp[1], q.flow, q.camera.f, q.camera.B, q.camera.cx, q.camera.cy)
            dt = time.perf_counter() - t0
            if keep is not None:
                keep["s4"], keep["motion"], keep["point"], keep["valid"] = res
    finally:
        for b in blocks:
            b.close()
            b.unlink()
        for b in _SHM.values():
            b.close()
        _SHM.clear()
    return {"value": round(1.0 / dt, 5), "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": "one full 1242x375 D=128 frame, the oracle's functions over 4 cost volumes and "
                      "32 (pass, direction) paths in spawned workers",
            "seconds": round(dt, 2), "cpu_model": cpu_model()}


def run_reference(args, rank):
    """Reference arm: the CPU oracle as it stands, each step a 1242x24 band of
    the frame (all 4 SGM passes + combination), scaled to frames/s by area."""
    from oracle import oracle
    from paper_1801_04720_gb300 import synth
    oracle.build()
    q = synth.automotive(seed=args.seed)
    band = 24
    y0 = 160
    sl = slice(y0, y0 + band)
    imgs = [np.ascontiguousarray(im[sl]) for im in q.images()]
    flow = np.ascontiguousarray(q.flow[sl])

    def step():
        oracle.scene_flow(imgs, flow, q.camera.f, q.camera.B, q.camera.cx, q.camera.cy - y0,
                          D=D_MAX)

    for _ in range(max(args.warmup, 1)):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    frac = band / H_IMG
    value = frac / dt
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "frames/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int + f64 (CPU oracle)",
        "data": "synthetic (seeded automotive-shaped scenes; KITTI is not available)",
        "config": {"workload": WORKLOAD, "W": W_IMG, "H": H_IMG, "D": D_MAX,
                   "sample": f"1242x{band} band per step, scaled by area"},
        "cpu_baseline": {"value": round(value, 5), "unit": "frames/s", "cores": 1,
                         "kind": "oracle", "sample": f"1242x{band} band per step, 1 thread"},
        "e2e": {"value": round(value, 5), "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


import numpy as np  # noqa: E402  (used by the reference arm)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank)), flush=True)
        return
    result, q = run_ours(args, world, rank, local)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            result["cpu_baseline"] = cpu_baseline(q)
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
