"""Training the snapshot codec on snapshots the propagator itself generates.

The training set comes from forward modelling (store-all snapshots every
``every`` steps) on seeded smooth random velocity models; the network is
trained by the library's own tensor-core forward and backward kernels and
Adam (``codec.train_step``). Nothing here computes the method: the
propagation, the codec and the optimiser all run in librtm.
"""
from __future__ import annotations

import math
import time
from typing import Optional

import numpy as np
import torch

import rtm_inputs

from . import codec
from . import (alloc_workspace, forward, make_params, model_prep, snapshot)


def training_snapshots(n_models: int = 64, size: int = 192, nb: int = 32, nt: int = 1200,
                       every: int = 100, first: int = 200, f0: float = 20.0, seed0: int = 1000,
                       dx: float = 10.0, vmin: float = 1500.0, vmax: float = 4500.0,
                       device="cuda") -> torch.Tensor:
    """Snapshots [S][size][size][size] (float32, on the device) of forward
    modelling on ``n_models`` seeded smooth random models (sigma 8 cells,
    [vmin, vmax]); one surface source per model at a seeded position; the
    snapshots at the multiples of ``every`` from ``first`` to ``nt``."""
    dt = rtm_inputs.courant_dt(dx, vmax)
    rng = np.random.Generator(np.random.PCG64(seed0))
    steps = list(range(every * max(1, -(-first // every)), nt + 1, every))
    out = torch.empty((n_models * len(steps), size, size, size), dtype=torch.float32,
                      device=device)
    k = 0
    for i in range(n_models):
        src = (int(rng.integers(size // 4, 3 * size // 4)),
               int(rng.integers(size // 4, 3 * size // 4)), 4)
        p = make_params(size, size, size, nb, 4, nt, dx, dt, f0, 1.0 / f0, src, 1,
                        storage="all", image_every=every)
        ws = alloc_workspace(p, device)
        v = rtm_inputs.smooth_random_velocity(size, size, size, 8.0, vmin, vmax,
                                              seed=seed0 + 1 + i, device=device)
        c = model_prep(p, v.contiguous(), ws)
        rec = torch.tensor([[size // 2, size // 2, 2]], dtype=torch.int32, device=device)
        forward(p, c, rec, ws)
        for m in steps:
            snapshot(p, ws, m, out=out[k])
            k += 1
        del ws, c, v
    return out


def train(data: torch.Tensor, steps: int = 1500, batch: int = 4, lr: float = 1e-3,
          lr_min: float = 5e-5, seed: int = 0, params: Optional[torch.Tensor] = None,
          log_every: int = 0):
    """Adam on random mini-batches of ``data`` with a cosine learning-rate
    decay from ``lr`` to ``lr_min``. Returns (params, losses)."""
    dev = data.device
    if params is None:
        params = torch.from_numpy(
            rtm_inputs.ae_flat(rtm_inputs.ae_init_params(seed)).astype(np.float32)).to(dev)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    ws = codec.alloc_workspace(tuple(data.shape[1:]), dev)
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    t0 = time.time()
    for step in range(1, steps + 1):
        idx = torch.randint(0, data.shape[0], (batch,), generator=g)
        xb = data[idx.to(dev)].contiguous()
        lr_t = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * (step - 1) / steps))
        codec.train_step(params, m, v, step, lr_t, xb, ws, loss=loss)
        if log_every and (step % log_every == 0 or step == 1):
            losses.append((step, float(loss.item()), time.time() - t0))
    if not losses or losses[-1][0] != steps:
        losses.append((steps, float(loss.item()), time.time() - t0))
    return params, losses


def reconstruction_error(params: torch.Tensor, snaps: torch.Tensor) -> float:
    """Relative L2 error of encode + decode over a set of snapshots."""
    ws = codec.alloc_workspace(tuple(snaps.shape[1:]), snaps.device)
    num = den = 0.0
    for s in snaps:
        lat, sc = codec.encode(params, s, ws)
        r = codec.decode(params, lat, sc, ws)
        num += float(((r - s) ** 2).sum())
        den += float((s * s).sum())
    return math.sqrt(num / max(den, 1e-300))
