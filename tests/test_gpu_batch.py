"""Batched quadruples of uneven size and disparity range (one persistent sweep
launch per kernel shape, optional CUDA-graph replay): every output bit-equal
to per-instance sf_scene_flow runs, and one small item checked against the
oracle; tuned sweep shapes give identical results."""
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


def _scene(sf, q):
    return {"left_t": to_dev(q.left_t), "right_t": to_dev(q.right_t), "left_t1": to_dev(q.left_t1),
            "right_t1": to_dev(q.right_t1), "flow": to_dev(q.flow), "D": q.D,
            "cam": sf.camera(q.camera.f, q.camera.B, q.camera.cx, q.camera.cy)}


SMALL = [(96, 64, 16), (130, 41, 48), (67, 53, 32), (200, 60, 64), (97, 40, 100), (130, 41, 128),
         (64, 48, 16), (160, 50, 192)]


def _quads(specs, seed0=0):
    out = []
    for k, (W, H, D) in enumerate(specs):
        disp = (2, max(3, D // 3), max(4, D - 5))
        out.append(synth.fronto_planes(W=W, H=H, D=D, disparities=disp, seed=seed0 + k))
    return out


def _compare(sf, quads, graph, repeats=1):
    import torch
    p = sf.params()
    scenes = [_scene(sf, q) for q in quads]
    outs = [sf.alloc_scene_flow_outputs(q.shape[1], q.shape[0], "cuda") for q in quads]
    items = sf.make_batch(scenes, outs)
    ws = torch.empty(sf.sf_batch_workspace_size(items, p), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream() if graph else torch.cuda.current_stream()
    for _ in range(repeats):
        for o in outs:
            for v in o.values():
                if v is not None:
                    v.fill_(0)
        torch.cuda.synchronize()
        sf.sf_batch_run(items, p, ws, graph=graph, stream=stream)
        torch.cuda.synchronize()
        for q, sc, o in zip(quads, scenes, outs):
            H, W = q.shape
            pq = sf.params(D=q.D)
            ref = sf.sf_scene_flow([sc["left_t"], sc["right_t"], sc["left_t1"], sc["right_t1"]],
                                   sc["flow"], pq, sc["cam"])
            for k in ("s4", "motion", "point", "valid", "D0", "D1"):
                a, b = to_np(o[k]), to_np(ref[k])
                assert np.array_equal(np.nan_to_num(a, nan=-9.0), np.nan_to_num(b, nan=-9.0)), (q.D, k)
    return outs


def test_batch_equals_per_instance(sf):
    _compare(sf, _quads(SMALL), graph=False)


def test_batch_graph_replay_equals_per_instance(sf):
    _compare(sf, _quads(SMALL, seed0=20), graph=True, repeats=3)
    sf.sf_batch_release_graphs()


def test_batch_with_wide_rows_equals_per_instance(sf):
    # 1242 x 192 and 900 x 256 distances per row exceed one CTA's shared memory
    _compare(sf, _quads([(1242, 24, 192), (96, 64, 16), (900, 20, 256)], seed0=40), graph=True)


def test_batch_small_item_against_oracle(sf, oracle_mod):
    quads = _quads([(64, 48, 16), (96, 64, 32)], seed0=7)
    outs = _compare(sf, quads, graph=False)
    q, o = quads[0], outs[0]
    r0 = oracle_mod.disparity(q.left_t, q.right_t, D=q.D)
    assert_nan_equal_close(to_np(o["D0"]), r0["disp"], SUBPIXEL_ATOL, "D0")


def test_batch_graph_needs_a_created_stream(sf):
    import torch
    quads = _quads([(64, 48, 16)])
    p = sf.params()
    sc = [_scene(sf, q) for q in quads]
    o = [sf.alloc_scene_flow_outputs(64, 48, "cuda")]
    items = sf.make_batch(sc, o)
    ws = torch.empty(sf.sf_batch_workspace_size(items, p), dtype=torch.uint8, device="cuda")
    null = type("S", (), {"cuda_stream": 0})()
    with pytest.raises(sf.SFError):
        sf.sf_batch_run(items, p, ws, graph=True, stream=null)


def test_batch_rejects_bad_items(sf):
    import ctypes
    import torch
    q = _quads([(64, 48, 16)])[0]
    sc = _scene(sf, q)
    o = sf.alloc_scene_flow_outputs(64, 48, "cuda")
    items = sf.make_batch([sc], [o])
    items[0].D = 0
    assert sf.sf_batch_workspace_size(items, sf.params()) == 0
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(sf.SFError):
        sf.sf_batch_run(items, sf.params(), ws)


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("dc,halo", [(8, 8), (16, 8), (16, 16), (8, 16)])
def test_tuned_shapes_are_bit_identical(sf, dc, halo, order):
    quads = _quads([(130, 41, 64), (97, 40, 128)], seed0=40)
    base = [_scene(sf, q) for q in quads]
    ref = [sf.sf_scene_flow([s["left_t"], s["right_t"], s["left_t1"], s["right_t1"]], s["flow"],
                            sf.params(D=q.D), s["cam"]) for s, q in zip(base, quads)]
    sf.sf_set_sweep_schedule(33, 128, dc, halo, order)   # every provided shape covers this class
    try:
        got = [sf.sf_scene_flow([s["left_t"], s["right_t"], s["left_t1"], s["right_t1"]], s["flow"],
                                sf.params(D=q.D), s["cam"]) for s, q in zip(base, quads)]
    finally:
        sf.sf_set_sweep_shape(33, 128, 0, 0)
    for a, b in zip(got, ref):
        for k in ("valid", "D0", "D1", "s4"):
            x, y = to_np(a[k]), to_np(b[k])
            assert np.array_equal(np.nan_to_num(x, nan=-9.0), np.nan_to_num(y, nan=-9.0)), k


def _oracle_item(args):
    from oracle import oracle
    q = args
    c = q.camera
    return oracle.scene_flow(q.images(), q.flow, c.f, c.B, c.cx, c.cy, D=q.D)


def test_graph_replayed_mixed_batch_every_item_against_oracle(sf):
    """A batch mixing D = 16, 64 and 192 (three kernel shapes, three sweep
    launches) and a row too wide for one CTA's distance band, replayed from
    its CUDA graph three times: every item's D0, D1, validity, S4, motion and
    point against the oracle's whole path, element by element (integers and
    masks exact, subpixel within 1e-4 px, scene flow within 1e-5 relative)."""
    import multiprocessing as mp
    from gpu_helpers import assert_sceneflow_close
    quads = _quads([(96, 64, 16), (130, 41, 64), (200, 30, 192), (1242, 12, 192), (67, 53, 64)], seed0=90)
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(quads)) as pool:
        refs = pool.map(_oracle_item, quads)
    outs = _compare(sf, quads, graph=True, repeats=3)
    sf.sf_batch_release_graphs()
    for q, o, r in zip(quads, outs, refs):
        assert_nan_equal_close(to_np(o["D0"]), r["t0"]["disp"], SUBPIXEL_ATOL, f"D0 D={q.D}")
        assert_nan_equal_close(to_np(o["D1"]), r["t1"]["disp"], SUBPIXEL_ATOL, f"D1 D={q.D}")
        got = {k: to_np(o[k]) for k in ("s4", "motion", "point", "valid")}
        assert_sceneflow_close(got, r["s4"], r["motion"], r["point"], r["valid"])
        assert r["valid"].sum() > 0


def test_batch_in_waves_equals_one_wave(sf):
    """A wave limit bounds the batch workspace; the outputs stay bit-identical
    (with and without graph replay)."""
    import torch
    quads = _quads([(96, 64, 16), (130, 41, 64), (160, 30, 192), (67, 53, 64), (200, 60, 32)], seed0=70)
    p = sf.params()
    scenes = [_scene(sf, q) for q in quads]
    ref = _compare(sf, quads, graph=False)
    full = sf.sf_batch_workspace_size(sf.make_batch(scenes, [sf.alloc_scene_flow_outputs(
        q.shape[1], q.shape[0], "cuda") for q in quads]), p)
    try:
        sf.sf_set_batch_wave_limit(full // 3)
        outs = [sf.alloc_scene_flow_outputs(q.shape[1], q.shape[0], "cuda") for q in quads]
        items = sf.make_batch(scenes, outs)
        capped = sf.sf_batch_workspace_size(items, p)
        assert capped < full
        ws = torch.empty(capped, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.Stream()
        for graph in (False, True, True):
            for o in outs:
                for v in o.values():
                    if v is not None:
                        v.fill_(0)
            sf.sf_batch_run(items, p, ws, graph=graph, stream=stream)
            torch.cuda.synchronize()
            for a, b in zip(outs, ref):
                for k in ("s4", "motion", "point", "valid", "D0", "D1"):
                    x, y = to_np(a[k]), to_np(b[k])
                    assert np.array_equal(np.nan_to_num(x, nan=-9.0), np.nan_to_num(y, nan=-9.0)), k
    finally:
        sf.sf_set_batch_wave_limit(0)
        sf.sf_batch_release_graphs()


@pytest.mark.parametrize("order", [0, 1, 2])
def test_batch_under_every_scheduling_order(sf, order):
    """The batch's descriptor tables follow the scheduling order of each class
    (one launch per scan order, or both in one launch): bit-equal to
    per-instance runs under every order, graph replay included."""
    quads = _quads([(96, 64, 16), (130, 41, 64), (160, 30, 192), (97, 40, 100), (200, 60, 128)], seed0=80 + order)
    try:
        sf.sf_set_sweep_schedule(1, 256, 16, 8, order)
    except sf.SFError:
        sf.sf_set_sweep_schedule(33, 256, 16, 8, order)
        sf.sf_set_sweep_schedule(1, 32, 8, 8, order)
    try:
        _compare(sf, quads, graph=True, repeats=2)
    finally:
        sf.sf_set_sweep_shape(1, 256, 0, 0)
        sf.sf_set_sweep_shape(33, 256, 0, 0)
        sf.sf_set_sweep_shape(1, 32, 0, 0)
        sf.sf_batch_release_graphs()
