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


def test_per_mode_slab_heights_are_checked_on_the_host():
    import paper_1603_03971_gb300 as rtm

    rtm.set_tuning_mode(4, "fwd", 48)
    rtm.set_tuning_mode(8, "bwd_image", 0)
    rtm.set_tuning(4, 0, 0)  # clears the per-mode heights of radius 4
    from paper_1603_03971_gb300 import _lib

    for args in ((5, 0, 16), (4, 5, 16), (4, 7, 16), (4, 0, -1), (4, 9, 16)):
        with pytest.raises(_lib.RtmError):
            _lib.call("rtm_set_tuning_mode", *args)


@pytest.mark.gpu
def test_tune_stencil_picks_the_fastest_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    choice = autotune.tune_stencil(4, (104, 104, 104), steps=6, cache_path=path)
    trials = {tuple(int(x) for x in k.split("/")): v for k, v in choice["trials"].items()}
    assert {v for v, _ in trials} == {1, 2, 3}  # vector loads, TMA 16-row and 8-row tiles
    assert (choice["variant"], choice["zchunk"]) == min(trials, key=trials.get)
    # the slab height of each mode is the fastest of that mode's launches
    # within the chosen variant
    tm = {tuple(int(x) for x in k.split("/")): v for k, v in choice["trials_modes"].items()}
    assert set(choice["zchunk_modes"]) == {"fwd", "fwd_snap", "bwd_image"}
    for mode, zc in choice["zchunk_modes"].items():
        t = {z: m[mode] for (v, z), m in tm.items() if v == choice["variant"]}
        assert zc == min(t, key=t.get)
    cached = json.load(open(path))
    assert any(v["zchunk"] == choice["zchunk"] for v in cached.values())
    # the second call is served from the cache
    assert autotune.tune_stencil(4, (104, 104, 104), cache_path=path) == choice


@pytest.mark.gpu
def test_tune_batch_sweeps_tiles_and_slabs(tmp_path):
    import torch

    import paper_1603_03971_gb300 as rtm
    from paper_1603_03971_gb300 import batch as B

    path = str(tmp_path / "tune.json")
    nz, ny, nx = 48, 40, 56
    p = rtm.make_params(nx, ny, nz, 4, 8, 8, 10.0, 6e-4, 25.0, 0.04, (0, 0, 0), 0,
                        storage="ckpt", ckpt_every=4)
    aps = [B.Aperture(0, 0, 0, 40, 32, 32, 20, 16, 3, 2),
           B.Aperture(8, 4, 8, 48, 36, 40, 24, 18, 4, 2)]
    vel = torch.full((nz, ny, nx), 2500.0, device="cuda")
    choice = autotune.tune_batch(p, aps, vel, nt=4, cache_path=path)
    trials = {tuple(int(x) for x in k.split("/")): v for k, v in choice["trials"].items()}
    assert {v for v, _ in trials} == {2, 3}
    assert (0 in {z for _, z in trials})  # the per-wave automatic height
    assert (choice["variant"], choice["zchunk"]) == min(trials, key=trials.get)
    assert autotune.tune_batch(p, aps, vel, cache_path=path) == choice
