"""Host logic of the autotuner: the coordinate-descent search and the cache
(CPU only; the timing function is replaced by a synthetic cost)."""
import json

from paper_2609_08989_gb300 import autotune, scenes


def test_coordinate_descent_finds_separable_minimum(monkeypatch):
    target = {"block": 256, "refill": 4, "crossing_batch": 16}
    calls = []

    def fake_time(run, tune, reps):
        calls.append(dict(tune))
        full = {"block": 128, "refill": 8, "crossing_batch": 8, **tune}
        return 10.0 + sum(abs(full[k] - target[k]) for k in target) / 10.0

    monkeypatch.setattr(autotune, "_time", fake_time)
    space = {"block": [128, 256], "refill": [1, 2, 4, 8, 16], "crossing_batch": [4, 8, 16, 24]}
    best, ms, hist = autotune.search(lambda t: None, space, reps=1, sweeps=2)
    assert {k: best.get(k) for k in target} == target
    assert abs(ms - 10.0) < 1e-12
    assert len(hist) == len(calls)


def test_classes_and_cache_roundtrip(monkeypatch, tmp_path):
    assert autotune.workload_class(scenes.kerr_disk(8)) == "fp64"
    assert autotune.workload_class(scenes.kerr_disk_mixed(8)) == "mixed"
    assert autotune.workload_class(scenes.kerr_disk_mixed(8).replace(precision=scenes.MIXED_PAIR)) == "mixed_pair"
    assert autotune.workload_class(scenes.table_kerr(8)) == "table"
    assert autotune.workload_class(scenes.table_kerr(8).replace(precision=scenes.DOUBLE_FLOAT)) == "table_double_float"
    cache = tmp_path / "tuned.json"
    monkeypatch.setattr(autotune, "CACHE", str(cache))
    monkeypatch.setattr(autotune, "_cache", None)
    monkeypatch.setattr(autotune, "_device_key", lambda: "FakeGPU")
    autotune.record("fp64", {"refill": 4}, 1.0, 2.0, "w")
    assert json.load(open(cache))["FakeGPU"]["fp64"]["tune"] == {"refill": 4}
    assert autotune.cached(scenes.kerr_disk(8)) == {"refill": 4}
    assert autotune.cached(scenes.kerr_disk_mixed(8)) is None


def test_committed_cache_is_well_formed():
    data = autotune.load()
    for dev, classes in data.items():
        for cls, entry in classes.items():
            assert cls in autotune.SPACE
            for k, v in entry["tune"].items():
                assert k in autotune.SPACE[cls] and v in autotune.SPACE[cls][k]
            assert entry["ms"] <= entry["default_ms"] * 1.01


def test_batch_scenes_use_the_mixed_tolerance():
    for prec in (scenes.MIXED, scenes.MIXED_PAIR):
        assert all(s.rtol == scenes.MIXED_RTOL for s in scenes.batch_uneven(3, precision=prec))
    assert all(s.rtol == 1e-10 for s in scenes.batch_uneven(3, precision=scenes.FP64))
