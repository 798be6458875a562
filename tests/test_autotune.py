"""Autotuner: candidate slab heights and the JSON cache (host logic, no GPU),
and one real tuning run on the GPU."""
import json

import pytest

from paper_1603_03971_gb300 import autotune


def test_candidates_respect_the_queue_warmup_and_grid():
    for r in (4, 8):
        for NZ in (40, 104, 576):
            c = list(autotune.candidates(NZ, r))
            assert c == sorted(set(c))
            assert all(4 * r <= z <= NZ for z in c)
            assert NZ in c  # one slab for the whole column
    assert list(autotune.candidates(20, 8)) == []


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    assert autotune.load_cache(path) == {}
    autotune.save_cache({"k": {"zchunk": 48}}, path)
    assert autotune.load_cache(path) == {"k": {"zchunk": 48}}
    with open(path, "w") as f:
        f.write("{broken")
    assert autotune.load_cache(path) == {}


@pytest.mark.gpu
def test_tune_stencil_picks_the_fastest_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    choice = autotune.tune_stencil(4, (104, 104, 104), steps=6, cache_path=path)
    trials = {tuple(int(x) for x in k.split("/")): v for k, v in choice["trials"].items()}
    assert {v for v, _ in trials} == {1, 2}  # both plane-load variants timed
    assert (choice["variant"], choice["zchunk"]) == min(trials, key=trials.get)
    cached = json.load(open(path))
    assert any(v["zchunk"] == choice["zchunk"] for v in cached.values())
    # the second call is served from the cache
    assert autotune.tune_stencil(4, (104, 104, 104), cache_path=path) == choice
