"""Autotuner of the stencil launch shape.

For a stencil radius and a padded grid shape it times a short checkpointed
shot of ``rtm_shot`` (forward, recompute with snapshot writes, backward with
imaging: every kernel mode of a shot, whose best slab heights differ; the
per-launch timing of each mode picks a slab height per mode) or a
short ``rtm_batch`` (persistent multi-shot kernel) for each candidate z-slab
height (and plane-load variant where there is more than one), with CUDA
events after a warm-up, picks the fastest and caches the choice in a JSON
file keyed by (kind, radius, shape, GPU name). ``apply()`` installs a cached
or freshly tuned choice with ``rtm_set_tuning``.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, Iterable, Optional, Sequence, Tuple

import numpy as np
import torch

from . import _lib

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
_lock = threading.Lock()


def _key(kind: str, radius: int, shape: Sequence[int]) -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return "%s|r%d|%s|%s" % (kind, radius, "x".join(str(int(s)) for s in shape), name)


def load_cache(path: str = CACHE) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: Dict[str, dict], path: str = CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(NZ: int, radius: int) -> Iterable[int]:
    """Slab heights worth trying: powers of two and fractions of NZ, at least
    4 r planes (the register queue warm-up is 2 r planes per slab)."""
    out = set()
    for z in (16, 24, 32, 48, 64, 96, 128, 192, 256):
        if 4 * radius <= z <= NZ:
            out.add(z)
    for parts in (1, 2, 3, 4, 6, 8):
        z = -(-NZ // parts)
        if z >= 4 * radius:
            out.add(z)
    return sorted(out)


def _time_shot(p, c, rec, dobs, img, ws, steps: int):
    """Milliseconds per stencil step of a checkpointed shot (3 steps per time
    step: forward, recompute, backward), and milliseconds per launch of each
    stencil mode from the library's per-launch timing of a second shot."""
    from . import reset_stats, set_timing, shot, stats

    shot(p, c, rec, dobs, ws, img)  # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    shot(p, c, rec, dobs, ws, img)
    e1.record()
    torch.cuda.synchronize()
    total = e0.elapsed_time(e1) / (3 * steps)
    reset_stats()
    set_timing(True)
    try:
        shot(p, c, rec, dobs, ws, img)
    finally:
        set_timing(False)
    per_mode = {k: v["ms"] / v["launches"] for k, v in stats()["stencil"].items()
                if v["launches"] and v["ms"] > 0}
    return total, per_mode


def tune_stencil(radius: int, padded_shape: Tuple[int, int, int], steps: int = 12,
                 cache_path: str = CACHE, force: bool = False,
                 variants: Tuple[int, ...] = (1, 2, 3)) -> dict:
    """Best plane-load path and tile (1 vector loads; 2 TMA, 16-row tiles; 3
    TMA, 8-row tiles of 4-point vectors) and z-slab height for the
    single-shot stencil on a padded grid (NZ, NY, NX), timed on a
    constant-velocity model; trials are keyed "variant/zchunk"."""
    from . import RtmError, alloc_workspace, make_params, model_prep, set_tuning

    key = _key("stencil", radius, padded_shape)
    with _lock:
        cache = load_cache(cache_path)
    if key in cache and not force:
        return cache[key]
    NZ, NY, NX = padded_shape
    nb = 4
    p = make_params(NX - 2 * nb, NY - 2 * nb, NZ - 2 * nb, nb, radius, steps, 10.0, 6e-4, 20.0,
                    0.05, (1, 1, 1), 1, storage="ckpt", ckpt_every=max(1, steps // 2))
    ws = alloc_workspace(p)
    v = torch.full((p.nz, p.ny, p.nx), 3000.0, device="cuda")
    c = model_prep(p, v, ws)
    rec = torch.zeros((1, 3), dtype=torch.int32, device="cuda")
    dobs = torch.zeros((steps, 1), device="cuda")
    img = torch.zeros((p.nz, p.ny, p.nx), device="cuda")
    results, modes = {}, {}
    try:
        for variant in variants:
            for zc in candidates(NZ, radius):
                try:
                    set_tuning(radius, zc, variant)
                    results[(variant, zc)], modes[(variant, zc)] = _time_shot(
                        p, c, rec, dobs, img, ws, steps)
                except RtmError:
                    continue  # a variant this driver cannot run
    finally:
        set_tuning(radius, 0, 0)
    best = min(results, key=results.get)
    # within the best variant, the fastest slab height of each mode (its
    # launches move different bytes per point and balance differently)
    per_mode = {}
    for mode in ("fwd", "fwd_snap", "bwd_image"):
        t = {zc: m[mode] for (v, zc), m in modes.items() if v == best[0] and mode in m}
        if t:
            per_mode[mode] = int(min(t, key=t.get))
    choice = {"zchunk": int(best[1]), "variant": int(best[0]), "ms_per_step": results[best],
              "zchunk_modes": per_mode,
              "trials": {"%d/%d" % k: v for k, v in results.items()},
              "trials_modes": {"%d/%d" % k: v for k, v in modes.items()}}
    with _lock:
        cache = load_cache(cache_path)
        cache[key] = choice
        save_cache(cache, cache_path)
    return choice


def tune_batch(p, apertures, vel: torch.Tensor, nt: int = 8, cache_path: str = CACHE,
               force: bool = False, variants: Tuple[int, ...] = (2, 3),
               budget: int = 0) -> dict:
    """Best tile (2: 16-row tiles, 3: 8-row tiles of the TMA kernel) and
    work-item slab height (0: the per-wave automatic height) of the
    persistent multi-shot kernel for a set of apertures, timed on a short
    run (nt steps) of the batch under the given device-memory budget; trials
    are keyed "variant/zchunk"."""
    from . import batch as B
    from . import set_tuning

    shape = (len(apertures), max(a.nz for a in apertures), max(a.ny for a in apertures),
             max(a.nx for a in apertures))
    key = _key("batch", p.radius, shape)
    with _lock:
        cache = load_cache(cache_path)
    if key in cache and not force:
        return cache[key]
    q = p.copy(nt=nt, ckpt_every=max(1, nt // 2))
    ws = B.alloc_workspace(q, apertures, budget)
    dobs = torch.zeros(B.data_size(q, apertures), device="cuda")
    img = torch.zeros(tuple(vel.shape), device="cuda")
    NZ = max(a.nz for a in apertures) + 2 * p.nb
    results = {}
    try:
        for variant in variants:
            set_tuning(p.radius, 0, variant)
            for zc in [0] + list(candidates(NZ, p.radius)):
                B.run(q, apertures, vel, dobs, img, ws, budget=budget, zchunk=zc)  # warm-up
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                B.run(q, apertures, vel, dobs, img, ws, budget=budget, zchunk=zc)
                e1.record()
                torch.cuda.synchronize()
                results[(variant, zc)] = e0.elapsed_time(e1)
    finally:
        set_tuning(p.radius, 0, 0)
        del ws, dobs, img
        torch.cuda.empty_cache()
    best = min(results, key=results.get)
    choice = {"zchunk": int(best[1]), "variant": int(best[0]), "ms": results[best],
              "trials": {"%d/%d" % k: v for k, v in results.items()}}
    with _lock:
        cache = load_cache(cache_path)
        cache[key] = choice
        save_cache(cache, cache_path)
    return choice


def apply(radius: int, padded_shape, tune_if_missing: bool = True,
          cache_path: str = CACHE) -> Optional[dict]:
    """Install the cached (or freshly tuned) stencil choice for this shape."""
    from . import set_tuning

    cache = load_cache(cache_path)
    choice = cache.get(_key("stencil", radius, padded_shape))
    if choice is None and tune_if_missing:
        choice = tune_stencil(radius, padded_shape, cache_path=cache_path)
    if choice is not None:
        set_tuning(radius, int(choice["zchunk"]), int(choice.get("variant", 0)))
        from . import set_tuning_mode

        for mode, zc in choice.get("zchunk_modes", {}).items():
            set_tuning_mode(radius, mode, int(zc))
    return choice


__all__ = ["tune_stencil", "tune_batch", "apply", "candidates", "load_cache", "save_cache"]
del np, _lib
