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
from typing import Optional, Sequence

import numpy as np
import torch

import rtm_inputs

from . import codec
from . import (alloc_workspace, forward, make_params, model_prep, snapshot)


def training_snapshots(n_models: int = 64, size: int = 192, nb: int = 32, nt: int = 1200,
                       every: int = 100, first: int = 200, f0: float = 20.0, seed0: int = 1000,
                       dx: float = 10.0, vmin: float = 1500.0, vmax: float = 4500.0,
                       device="cuda", early: Sequence[int] = ()) -> torch.Tensor:
    """Snapshots [S][size][size][size] (float32, on the device) of forward
    modelling on ``n_models`` seeded smooth random models (sigma 8 cells,
    [vmin, vmax]); one surface source per model at a seeded position; the
    snapshots at the steps in ``early`` and at the multiples of ``every``
    from ``first`` to ``nt``."""
    dt = rtm_inputs.courant_dt(dx, vmax)
    rng = np.random.Generator(np.random.PCG64(seed0))
    steps = sorted(set(int(m) for m in early if 1 <= m <= nt) |
                   set(range(every * max(1, -(-first // every)), nt + 1, every)))
    out = torch.empty((n_models * len(steps), size, size, size), dtype=torch.float32,
                      device=device)
    k = 0
    for i in range(n_models):
        src = (int(rng.integers(size // 4, 3 * size // 4)),
               int(rng.integers(size // 4, 3 * size // 4)), 4)
        step_every = math.gcd(*steps) if steps else every
        p = make_params(size, size, size, nb, 4, nt, dx, dt, f0, 1.0 / f0, src, 1,
                        storage="all", image_every=step_every)
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
          log_every: int = 0, init: str = "decimation"):
    """Adam on random mini-batches of ``data`` with a cosine learning-rate
    decay from ``lr`` to ``lr_min``. Without ``params`` training starts from
    ``init``: "decimation" (the network set to compute the non-learned 8x
    scheme, ``decimation_init``) or "random" (seeded He-style weights).
    Returns (params, losses)."""
    dev = data.device
    if params is None:
        flat = (decimation_init(seed) if init == "decimation"
                else rtm_inputs.ae_flat(rtm_inputs.ae_init_params(seed)))
        params = torch.from_numpy(flat.astype(np.float32)).to(dev)
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


def decimation_init(seed: int = 0) -> np.ndarray:
    """Initial codec parameters (flat, float32) under which the network
    computes the non-learned 8x scheme exactly, up to bfloat16 rounding:
    keep every other sample on each axis, reconstruct by linear interpolation
    along each axis. Training starts from that scheme instead of from noise.

    * E1 channels 0 / 1: +x and -x of the sample at the even corner of each
      2^3 patch (LeakyReLU(v) - LeakyReLU(-v) = 1.1 v recovers it).
    * Latent channels 0..7: the eight kept samples of each 4^3 block, one per
      parity (pz, py, px) of the half-resolution grid (E2's tap pz + 1).
    * D1 channels c and 8 + c (c = child parity (az, ay, ax)): +/- the linear
      interpolation of the kept samples at q and q + 1 on each axis for the
      child 2q + a; a transposed-convolution tap k reads latent parity p as
      sample q + d with (k, p) = (1, 0): d = 0, (1, 1): d = 1, (2, 1): d = 0,
      (0, 0): d = 1, each weighted 1 / 0 (a = 0, d = 0 / 1) or 1/2 (a = 1).
    * D2 maps the pair back to the child's sample.

    Channels that carry the scheme read nothing else. The remaining channels
    (E1 2..31, latent 8..15, D1 16..31) keep their seeded random weights;
    D2 reads them with weight zero, so the initial output is the scheme's,
    and training grows their share from there."""
    P = rtm_inputs.ae_init_params(seed)
    inv = 1.0 / 1.1
    W1, W2, W3, W4 = P["W1"], P["W2"], P["W3"], P["W4"]
    W1[0:2] = 0.0
    W1[0, 0, 0, 0] = 1.0
    W1[1, 0, 0, 0] = -1.0
    W2[0:8] = 0.0
    for pz in range(2):
        for py in range(2):
            for px in range(2):
                o = 4 * pz + 2 * py + px
                W2[o, pz + 1, py + 1, px + 1, 0] = inv
                W2[o, pz + 1, py + 1, px + 1, 1] = -inv
    # per axis: weight of (tap k, latent parity p) for child parity a
    def w_axis(a, k, p):
        d = {(1, 0): 0, (1, 1): 1, (2, 1): 0, (0, 0): 1}.get((k, p))
        if d is None:
            return 0.0
        return 0.5 if a == 1 else (1.0 if d == 0 else 0.0)

    W3[0:16] = 0.0
    for az in range(2):
        for ay in range(2):
            for ax in range(2):
                c = 4 * az + 2 * ay + ax
                for kz in range(4):
                    for ky in range(4):
                        for kx in range(4):
                            for pz in range(2):
                                for py in range(2):
                                    for px in range(2):
                                        w = (w_axis(az, kz, pz) * w_axis(ay, ky, py) *
                                             w_axis(ax, kx, px))
                                        i = 4 * pz + 2 * py + px
                                        W3[c, kz, ky, kx, i] = w
                                        W3[8 + c, kz, ky, kx, i] = -w
    W4[...] = 0.0
    for az in range(2):
        for ay in range(2):
            for ax in range(2):
                c = 4 * az + 2 * ay + ax
                W4[az, ay, ax, c] = inv
                W4[az, ay, ax, 8 + c] = -inv
    for b in ("b1", "b2", "b3", "b4"):
        P[b][...] = 0.0
    return rtm_inputs.ae_flat(P).astype(np.float32)
