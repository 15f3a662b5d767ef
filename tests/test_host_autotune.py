"""Host logic of the autotuner (no GPU): the JSON cache, workload keys and the pick."""
import json
import os

import pytest

torch = pytest.importorskip("torch")

from paper_2601_17354_gb300 import autotune as A


def test_cache_round_trip_keeps_other_entries(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert A._load(path) == {}
    A._store(path, "k1", {"fwd": [2, 256], "bwd": [2, 128]})
    A._store(path, "k2", {"tile": 8})
    data = A._load(path)
    assert data == {"k1": {"fwd": [2, 256], "bwd": [2, 128]}, "k2": {"tile": 8}}
    A._store(path, "k1", {"fwd": [4, 64], "bwd": [4, 64]})
    assert A._load(path)["k1"] == {"fwd": [4, 64], "bwd": [4, 64]}
    assert A._load(path)["k2"] == {"tile": 8}
    # the write goes through a temporary file that is renamed over the cache
    assert [f for f in os.listdir(tmp_path / "sub") if ".tmp" in f] == []


def test_corrupt_or_missing_cache_reads_as_empty(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert A._load(str(path)) == {}
    A._store(str(path), "k", {"tile": 16})
    assert json.loads(path.read_text()) == {"k": {"tile": 16}}
    assert A._load(str(tmp_path / "absent.json")) == {}


def test_cache_path_prefers_argument_then_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("PGS_AUTOTUNE_CACHE", str(tmp_path / "env.json"))
    assert A._cache_path(None) == str(tmp_path / "env.json")
    assert A._cache_path(str(tmp_path / "arg.json")) == str(tmp_path / "arg.json")
    monkeypatch.delenv("PGS_AUTOTUNE_CACHE")
    assert A._cache_path(None) == A.DEFAULT_CACHE


def test_workload_key_classes():
    # resolutions are a set (order and repeats do not matter), Gaussian counts a power-of-two class
    k1 = A.workload_key("batch", ["1280x720", "640x480", "1280x720"], 200_000, 3)
    k2 = A.workload_key("batch", ["640x480", "1280x720"], 190_000, 3)  # log2 17.5 .. 18.5 -> 18
    assert k1 == k2
    assert k1.split("|")[1:] == ["batch", "1280x720+640x480", "N~2^18", "sh3"]
    assert A.workload_key("batch", ["640x480"], 200_000, 3) != k1
    assert A.workload_key("single", ["1280x720", "640x480"], 200_000, 3) != k1
    assert A.workload_key("batch", ["1280x720", "640x480"], 500_000, 3) != k1
    assert A.workload_key("batch", ["1280x720", "640x480"], 200_000, 1) != k1
    assert A.workload_key("batch", ["1x1"], 0, 0).split("|")[3] == "N~2^0"
    assert A.resolution_class(1920, 1080) == "1920x1080"


def test_pick_takes_the_fastest():
    assert A.pick({(2, 256): 0.52, (4, 64): 0.49, (1, 128): 0.61}) == (4, 64)
    assert A.pick({8: 1.3}) == 8


def test_variants_apply_sets_both_kernels():
    calls = []

    class FakeRasterizer:
        def set_variants(self, fwd, bwd):
            calls.append((fwd, bwd))

    v = A.Variants(fwd=(2, 256), bwd=(4, 128), ms=0.75)
    v.apply(FakeRasterizer())
    assert calls == [((2, 256), (4, 128))]
    with pytest.raises(Exception):
        v.fwd = (1, 64)  # frozen
