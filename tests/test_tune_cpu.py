"""The autotuner's cache on the CPU: a fake matrix stands in for the device
calls (its tune() returns a fixed winner, set_config records what it is
given), so that the key, the hit and miss paths, retuning and the file
handling are checked without a GPU."""
import json

import pytest

from paper_1411_2377_gb300 import tune


class FakeMatrix:
    def __init__(self, prec=256, row_hist=(0, 10, 120, 40)):
        self.prec = prec
        self.row_hist = list(row_hist)
        self.tuned = []
        self.set = []

    def tune(self, mode, reps):
        self.tuned.append((mode, reps))
        tpb = 128 if mode == "ordered" else 64
        return {"threads_per_block": tpb, "variant": 13 if mode == "ordered" else 9,
                "carveout": -1, "ms": 0.25}

    def set_config(self, mode, tpb, variant, carve):
        self.set.append((mode, tpb, variant, carve))


@pytest.fixture(autouse=True)
def one_gpu_name(monkeypatch):
    monkeypatch.setattr(tune, "_gpu_name", lambda: "GB300 (test)")


def test_miss_then_hit(tmp_path):
    cache = str(tmp_path / "sub" / "tune.json")
    A = FakeMatrix()
    out = tune.autotune(A, reps=3, cache=cache)
    assert A.tuned == [("ordered", 3), ("exact", 3)] and A.set == []
    assert not out["ordered"]["cached"] and out["ordered"]["ms"] == 0.25
    stored = json.load(open(cache))
    assert len(stored) == 2
    B = FakeMatrix()  # same precision and row-length histogram: same key
    out = tune.autotune(B, cache=cache)
    assert B.tuned == []
    assert B.set == [("ordered", 128, 13, -1), ("exact", 64, 9, -1)]
    assert out["exact"]["cached"] and out["exact"]["ms"] is None


def test_retune_times_again(tmp_path):
    cache = str(tmp_path / "tune.json")
    tune.autotune(FakeMatrix(), modes=("ordered",), cache=cache)
    A = FakeMatrix()
    out = tune.autotune(A, modes=("ordered",), cache=cache, retune=True)
    assert A.tuned == [("ordered", 5)] and A.set == []
    assert not out["ordered"]["cached"]


def test_key_separates_precision_mode_and_histogram_but_not_small_count_changes():
    base = FakeMatrix()
    k = tune.signature(base, "ordered")
    assert tune.signature(base, "exact") != k
    assert tune.signature(FakeMatrix(prec=512), "ordered") != k
    assert tune.signature(FakeMatrix(row_hist=(0, 10, 120, 40, 1)), "ordered") != k
    # counts are rounded to two significant digits: 120 -> 121 keeps the key
    assert tune.signature(FakeMatrix(row_hist=(0, 10, 121, 40)), "ordered") == k


def test_unreadable_cache_is_treated_as_empty(tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text("{not json")
    A = FakeMatrix()
    tune.autotune(A, modes=("exact",), cache=str(cache))
    assert A.tuned == [("exact", 5)]
    assert list(json.load(open(cache)).values()) == [
        {"threads_per_block": 64, "variant": 9, "carveout": -1}]
    assert [p.name for p in tmp_path.iterdir()] == ["tune.json"]  # no temporary left


def test_no_cache_writes_nothing(tmp_path, monkeypatch):
    monkeypatch.chdir(tmp_path)
    A = FakeMatrix()
    tune.autotune(A, cache=None)
    assert len(A.tuned) == 2 and list(tmp_path.iterdir()) == []
