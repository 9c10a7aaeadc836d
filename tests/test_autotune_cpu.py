"""Host side of the sweep-shape autotuner (no GPU): installing a tuned
choice, rejecting shapes the library does not provide, and the cache key."""
import json

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1801_04720_gb300 import _lib, build
    build.build()
    _lib.load()
    yield _lib
    for lo, hi in [(1, 32), (33, 64), (65, 128), (129, 256)]:
        _lib.sf_set_sweep_shape(lo, hi, 0, 0)
        _lib.sf_set_learned_sweep_schedule(lo, hi, 0, 0, 0)


def test_apply_installs_every_class(lib):
    from paper_1801_04720_gb300 import autotune
    res = {"classes": [{"lo": 33, "hi": 64, "dc": 8, "halo": 8, "order": 1},
                       {"lo": 65, "hi": 128, "dc": 16, "halo": 16, "order": 0},
                       {"lo": 129, "hi": 256, "dc": 16, "halo": 8}]}      # no order: 0
    assert autotune.apply(res) == 3
    for c in res["classes"]:
        lib.sf_set_sweep_shape(c["lo"], c["hi"], 0, 0)


def test_apply_installs_the_learned_table(lib):
    from paper_1801_04720_gb300 import autotune
    res = {"classes": [{"lo": 65, "hi": 128, "dc": 16, "halo": 8, "order": 1}],
           "learned": [{"lo": 65, "hi": 128, "dc": 16, "halo": 8, "order": 2},
                       {"lo": 129, "hi": 256, "dc": 16, "halo": 8, "order": 0}]}
    assert autotune.apply(res) == 3
    lib.sf_set_sweep_shape(65, 128, 0, 0)
    for c in res["learned"]:
        lib.sf_set_learned_sweep_schedule(c["lo"], c["hi"], 0, 0, 0)


@pytest.mark.parametrize("args", [(1, 32, 4, 16, 1), (65, 128, 8, 12, 1), (200, 100, 8, 16, 1),
                                  (129, 257, 16, 8, 1), (65, 128, 16, 8, 3), (65, 128, 16, 8, -1)])
def test_learned_table_rejects_what_the_plain_table_rejects(lib, args):
    with pytest.raises(lib.SFError):
        lib.sf_set_sweep_schedule(*args)
    with pytest.raises(lib.SFError):
        lib.sf_set_learned_sweep_schedule(*args)


def test_learned_table_holds_sixteen_classes(lib):
    for d in range(1, 17):
        lib.sf_set_learned_sweep_schedule(d, d, 8, 8, 1)
    with pytest.raises(lib.SFError):      # full, while the plain table is not
        lib.sf_set_learned_sweep_schedule(17, 17, 8, 8, 1)
    lib.sf_set_sweep_schedule(17, 17, 8, 8, 1)
    lib.sf_set_sweep_shape(17, 17, 0, 0)
    for d in range(1, 17):
        lib.sf_set_learned_sweep_schedule(d, d, 0, 0, 0)
    lib.sf_set_learned_sweep_schedule(17, 17, 8, 8, 1)
    lib.sf_set_learned_sweep_schedule(17, 17, 0, 0, 0)


@pytest.mark.parametrize("lo,hi,dc,halo", [(1, 32, 4, 16), (65, 128, 8, 12), (200, 100, 8, 16),
                                          (0, 32, 8, 16), (129, 257, 16, 8)])
def test_unsupported_shapes_are_rejected(lib, lo, hi, dc, halo):
    with pytest.raises(lib.SFError):
        lib.sf_set_sweep_shape(lo, hi, dc, halo)


@pytest.mark.parametrize("order", [-1, 3, 7])
def test_unknown_scheduling_orders_are_rejected(lib, order):
    with pytest.raises(lib.SFError):
        lib.sf_set_sweep_schedule(65, 128, 16, 8, order)


def test_parse_key_round_trip():
    from paper_1801_04720_gb300 import autotune
    for dc, halo, order in autotune.CANDIDATES:
        assert autotune.parse_key(f"{dc}x{halo}o{order}") == (dc, halo, order)


def test_every_candidate_is_a_built_shape(lib):
    from paper_1801_04720_gb300 import autotune
    for lo, hi in autotune.DEFAULT_CLASSES:
        ok = 0
        for dc, halo, order in autotune.CANDIDATES:
            try:
                lib.sf_set_sweep_schedule(lo, hi, dc, halo, order)
                ok += 1
            except lib.SFError:
                pass
            lib.sf_set_sweep_shape(lo, hi, 0, 0)
        assert ok >= 1, (lo, hi)     # D > 128 has one built shape (16 disparities, halo 8)


def test_cache_is_keyed_by_gpu_and_size(tmp_path):
    from paper_1801_04720_gb300 import autotune
    path = tmp_path / "tune.json"
    res = {"gpu": "GPU-A", "W": 1242, "H": 375,
           "classes": [{"lo": 65, "hi": 128, "dc": 8, "halo": 16, "order": 1}]}
    path.write_text(json.dumps(res))
    assert autotune.cached(str(path), "GPU-A", 1242, 375) == res
    assert autotune.cached(str(path), "GPU-B", 1242, 375) is None
    assert autotune.cached(str(path), "GPU-A", 640, 480) is None
    assert autotune.cached(str(tmp_path / "missing.json"), "GPU-A", 1242, 375) is None
    # a cache written before the scheduling order was tuned is stale
    old = {"gpu": "GPU-A", "W": 1242, "H": 375, "classes": [{"lo": 65, "hi": 128, "dc": 8, "halo": 16}]}
    path.write_text(json.dumps(old))
    assert autotune.cached(str(path), "GPU-A", 1242, 375) is None
    path.write_text("{not json")
    assert autotune.cached(str(path), "GPU-A", 1242, 375) is None


def test_tune_table_picks_the_fastest_and_drops_each_trial(monkeypatch):
    """The per-table search with a fake timer: every built candidate is
    installed once, dropped after its timing, and the fastest is kept."""
    from paper_1801_04720_gb300 import autotune, synth
    monkeypatch.setattr(synth, "fronto_planes", lambda **kw: None)
    calls = []

    def setter(lo, hi, dc, halo, order):
        calls.append((lo, hi, dc, halo, order))
        if (dc, halo) == (8, 8) and order == 2:
            raise autotune._lib.SFError("sf_set_sweep_schedule", 2)   # not built

    def timer(q, D):
        dc, halo, order = calls[-1][2:]
        return 1.0 + 0.1 * order + (0.05 if dc == 8 else 0.0) + (0.01 if halo == 16 else 0.0)

    out = autotune._tune_table([(65, 128)], 1242, 375, 0, timer, setter)
    assert len(out) == 1
    best = out[0]
    assert (best["dc"], best["halo"], best["order"]) == (16, 8, 0)
    assert "8x8o2" not in best["candidates_ms"]
    assert len(best["candidates_ms"]) == len(autotune.CANDIDATES) - 1
    # every trial is followed by dropping the class again
    trials = [c for c in calls if c[2] != 0]
    drops = [c for c in calls if c[2] == 0]
    assert len(drops) == len(trials) - 1 and all(c[:2] == (65, 128) for c in calls)
