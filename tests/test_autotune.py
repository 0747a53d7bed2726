"""Host logic of the autotuner and of the tile settings (no GPU)."""
import json

import pytest

import bench
from paper_2210_16998_gb300 import autotune, tpg


def test_bitset_words_classes():
    # 32 vertices per word, rounded up to the instantiated widths
    assert [autotune.bitset_words(n) for n in (1, 32, 33, 96, 97, 160, 161, 200, 257, 4096)] == \
        [1, 1, 2, 3, 4, 5, 6, 8, 16, 128]
    with pytest.raises(ValueError):
        autotune.bitset_words(4097)


class _Cfg:
    def __init__(self, n):
        self.n = n


def test_tune_uses_a_cached_tile_without_measuring(tmp_path, monkeypatch):
    path = str(tmp_path / "tuned.json")
    autotune.save_cache({"W5": {"shape": [512, 2, 2], "ms": 1.0}}, path)

    def no_measuring(*a, **k):
        raise AssertionError("a cached width must not be measured again")

    monkeypatch.setattr(autotune, "measure_shapes", no_measuring)
    tile, entry = autotune.tune(cfgs=[_Cfg(150)], path=path)
    assert tile == (512, 2, 2) and entry["ms"] == 1.0


def test_tune_measures_and_caches_the_fastest_tile(tmp_path, monkeypatch):
    path = str(tmp_path / "tuned.json")
    # an entry of the older two-number form is measured again
    autotune.save_cache({"W5": {"shape": [256, 1], "ms": 9.0}}, path)
    fake = {(256, 1, 1): 7.0, (1024, 1, 1): 5.5, (1024, 1, 2): 5.25, (512, 1, 1): 6.0}
    calls = []

    def measure(cfgs, reps=3):
        calls.append(len(cfgs))
        return 5, dict(fake)

    monkeypatch.setattr(autotune, "measure_shapes", measure)
    tile, entry = autotune.tune(cfgs=[_Cfg(150), _Cfg(20)], path=path)
    assert calls == [2]
    assert tile == (1024, 1, 2) and entry["ms"] == 5.25
    assert entry["all"]["1024x1/2"] == 5.25 and entry["all"]["256x1/1"] == 7.0
    with open(path) as f:
        stored = json.load(f)
    assert stored["W5"]["shape"] == [1024, 1, 2]
    # the stored entry is used from now on
    monkeypatch.setattr(autotune, "measure_shapes", lambda *a, **k: pytest.fail("measured twice"))
    assert autotune.tune(cfgs=[_Cfg(150)], path=path)[0] == (1024, 1, 2)


def test_parse_tile():
    assert bench.parse_tile("") is None
    assert bench.parse_tile("512,1") == (512, 1)
    assert bench.parse_tile("1024,1,2") == (1024, 1, 2)
    for bad in ("512", "1,2,3,4"):
        with pytest.raises(SystemExit):
            bench.parse_tile(bad)


def test_set_tile_applies_shape_and_split(monkeypatch):
    calls = []
    monkeypatch.setattr(tpg, "tpg_set_tile_shape", lambda cfg, b, i: calls.append(("shape", b, i)))
    monkeypatch.setattr(tpg, "tpg_set_work_split", lambda cfg, s: calls.append(("split", s)))
    tpg.set_tile(object(), (512, 2))
    tpg.set_tile(object(), (1024, 1, 2))
    assert calls == [("shape", 512, 2), ("split", 1), ("shape", 1024, 1), ("split", 2)]
