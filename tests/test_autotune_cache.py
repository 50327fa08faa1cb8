"""Autotuner cache (host logic, no GPU): keys, round trip, unreadable files."""
import json

import paper_1010_2592_gb300 as fa


def test_tune_key_names_lattice_precision_and_gpu():
    assert fa.tune_key((16, 16, 16, 32), "GPU X") == "16x16x16x32|f32|GPU X"
    assert fa.tune_key([8, 8, 8, 8], "g", "f32") != fa.tune_key([8, 8, 8, 16], "g", "f32")


def test_cache_round_trip_and_merge(tmp_path):
    path = str(tmp_path / "tune.json")
    assert fa.load_tune_cache(path) == {}
    fa.store_tune_cache(path, "a", {"shape": 2, "times_ms": [0.02, 0.01]})
    fa.store_tune_cache(path, "b", {"shape": 1, "times_ms": [0.1, 0.2]})
    data = fa.load_tune_cache(path)
    assert data == {"a": {"shape": 2, "times_ms": [0.02, 0.01]}, "b": {"shape": 1, "times_ms": [0.1, 0.2]}}
    with open(path) as f:
        assert json.load(f) == data


def test_unreadable_cache_reads_as_empty(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert fa.load_tune_cache(str(path)) == {}
    path.write_text("[1, 2]")
    assert fa.load_tune_cache(str(path)) == {}


def test_shape_names():
    assert (fa.SHAPE_AUTO, fa.SHAPE_WIDE, fa.SHAPE_NARROW) == (0, 1, 2)
