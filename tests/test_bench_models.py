"""bench.py's host-side models on CPU: the algorithmic byte counts behind the
roofline numbers, and the lookup of measured DRAM traffic, which must give
nothing once the kernel sources differ from those the capture was taken
with, or for a sweep shape that was not captured."""
import hashlib
import json

import pytest


def test_sweep_bytes_model():
    import bench
    N, D = 1242 * 375, 128
    # the partial sum of one scan order, uint16, written and read once per
    # pass: a launch per scan order does one of the two, a merged launch both
    assert bench.bytes_model("sgm_sweep", N, D, order=0) == 4 * 2 * N * D
    assert bench.bytes_model("sgm_sweep", N, D, order=0) == 476_928_000
    assert bench.bytes_model("sgm_sweep", N, D, order=1) == 4 * 4 * N * D
    assert bench.bytes_model("sgm_sweep", N, D) == 953_856_000
    # the horizontal paths' launch: the cost in, both uint8 path volumes out, per pass
    assert bench.bytes_model("aggregate", N, D) == 4 * 3 * N * D
    # order 2: the merged launch runs the horizontal paths too
    assert bench.bytes_model("sgm_sweep", N, D, order=2) == 4 * 4 * N * D + 4 * 3 * N * D
    assert bench.stage_bytes_model("sgm_sweep", N, D, order=2) == bench.bytes_model("sgm_sweep", N, D, order=2)


def test_frame_bytes_model_itemised():
    import bench
    N, D = 1000, 64
    items = {
        "partial sums, 4 passes x (write + read) x uint16": 4 * 2 * 2 * N * D,
        "images in": 4 * N,
        "census strings written and read": 4 * 8 * 2 * N,
        "winners of four passes written and read": 4 * 2 * 2 * N,
        "two disparity maps written and read": 2 * 4 * 2 * N,
        "flow in": 8 * N,
        "outputs (s4, motion, point, valid)": (16 + 12 + 12 + 1) * N,
    }
    assert bench.frame_bytes_model(N, D) == sum(items.values())


@pytest.fixture()
def fake_root(tmp_path, monkeypatch):
    import bench
    src = tmp_path / "k.cu"
    src.write_bytes(b"kernel v1")
    sha = hashlib.sha256(b"kernel v1").hexdigest()
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"sgm_sweep": {"by_shape": {"16x16": {"bytes_per_launch": 11}, "8x16": {"bytes_per_launch": 22}},
                         "sources": ["k.cu"], "sources_sha256": sha},
           "aggregate": {"bytes_per_launch": 33, "shape": "any", "sources": ["k.cu"], "sources_sha256": sha},
           "old": {"bytes_per_launch": 44, "shape": "16x16", "sources": ["k.cu"], "sources_sha256": sha}}
    (prof / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return src


def test_measured_traffic_by_shape(fake_root):
    import bench
    assert bench.measured_traffic("sgm_sweep", "16x16") == 11
    assert bench.measured_traffic("sgm_sweep", "8x16") == 22
    assert bench.measured_traffic("sgm_sweep", "16x8") is None
    assert bench.measured_traffic("aggregate") == 33
    assert bench.measured_traffic("old", "16x16") == 44
    assert bench.measured_traffic("old", "8x16") is None
    assert bench.measured_traffic("missing") is None


def test_measured_traffic_void_after_source_change(fake_root):
    import bench
    fake_root.write_bytes(b"kernel v2")
    assert bench.measured_traffic("sgm_sweep", "16x16") is None
    assert bench.measured_traffic("aggregate") is None


def test_all_cores_oracle_equals_the_oracle():
    """The all-cores baseline runs the oracle's own functions on independent
    units; its frame must be the single-thread oracle's frame."""
    import numpy as np
    import bench
    from oracle import oracle
    from paper_1801_04720_gb300 import synth
    q = synth.fronto_planes(seed=4)
    keep = {}
    r = bench.cpu_baseline_all_cores(q, cores=2, D=q.D, keep=keep)
    assert r["cores"] == 2 and r["value"] > 0 and r["cpu_model"]
    c = q.camera
    ref = oracle.scene_flow(q.images(), q.flow, c.f, c.B, c.cx, c.cy, D=q.D)
    assert np.array_equal(keep["valid"], ref["valid"])
    assert np.array_equal(keep["s4"], ref["s4"], equal_nan=True)
    assert np.array_equal(keep["motion"], ref["motion"], equal_nan=True)


def test_densify_bytes_model():
    import bench
    N = 1242 * 375
    # two maps: row pass read twice + written twice (16 N); back-projection 24 N in, 41 N out
    assert bench.densify_bytes_model(N) == 2 * 16 * N + 24 * N + 41 * N == 97 * N


def test_stage_bytes_model():
    import bench
    N, D = 1242 * 375, 128
    m = {k: bench.stage_bytes_model(k, N, D) for k in ("census", "cost", "aggregate", "sgm_sweep", "combine")}
    assert m["census"] == 4 * N + 4 * 8 * N
    assert m["cost"] == 4 * 8 * N + 4 * N * D                # two pairs, both references
    assert m["aggregate"] == 4 * (N * D + 2 * N * D)          # cost in, two path volumes out
    assert m["sgm_sweep"] == bench.bytes_model("sgm_sweep", N, D, order=1)
    assert m["combine"] == (2 + 2 + 4) * 2 * N + 8 * N + (4 + 4 + 16 + 12 + 12 + 1) * N
    assert bench.stage_bytes_model("features", N, D) is None
