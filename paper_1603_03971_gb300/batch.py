"""Batched multi-shot RTM on uneven apertures: binding of rtm_batch.

All shots of a wave run inside one persistent cooperative kernel launch that
balances their uneven tiles dynamically; every wave's work is captured into
one CUDA graph per call.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import torch

from ._lib import RtmParams, call, lib


class Aperture(ctypes.Structure):
    """Mirror of ``rtm_aperture``: origin and size of a shot's aperture in the
    full model, its source and its receiver plane in aperture coordinates."""

    _fields_ = [(n, ctypes.c_int32) for n in
                ("ox", "oy", "oz", "nx", "ny", "nz", "src_x", "src_y", "src_z", "rec_z")]


def _arr(apertures: Sequence[Aperture]):
    return (Aperture * len(apertures))(*apertures)


def workspace_size(p: RtmParams, apertures, budget: int = 0) -> int:
    n = lib().rtm_batch_workspace_size(ctypes.byref(p), len(apertures), _arr(apertures),
                                       ctypes.c_size_t(budget))
    if n == 0:
        raise ValueError("invalid batch: " + (lib().rtm_last_error() or b"").decode())
    return int(n)


def alloc_workspace(p: RtmParams, apertures, budget: int = 0, device="cuda") -> torch.Tensor:
    return torch.empty(workspace_size(p, apertures, budget), dtype=torch.uint8, device=device)


def data_size(p: RtmParams, apertures) -> int:
    """Floats of the concatenated per-shot data [nt][ny_s][nx_s]."""
    return sum(p.nt * a.nx * a.ny for a in apertures)


def run(p: RtmParams, apertures, vel: torch.Tensor, dobs: torch.Tensor, image: torch.Tensor,
        ws: torch.Tensor, data=None, budget: int = 0, zchunk: int = 0, stream=None):
    """RTM of every shot; images accumulate into ``image`` (full model)."""
    s = torch.cuda.current_stream() if stream is None else stream
    for t, name in ((vel, "vel"), (dobs, "dobs"), (image, "image")):
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA float32 tensor" % name)
    call("rtm_batch", ctypes.byref(p), len(apertures), _arr(apertures),
         ctypes.c_void_p(vel.data_ptr()), ctypes.c_void_p(dobs.data_ptr()),
         ctypes.c_void_p(data.data_ptr()) if data is not None else None,
         ctypes.c_void_p(image.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
         ctypes.c_size_t(ws.numel()), ctypes.c_size_t(budget), int(zchunk),
         ctypes.c_void_p(s.cuda_stream))
    return image


def set_wait(seconds: float = 20.0, poison_shot: int = -1):
    """Bound of the persistent kernel's inter-block waits; ``poison_shot``
    injects a wait that never completes (failure-path testing)."""
    call("rtm_batch_set_wait", ctypes.c_double(seconds), int(poison_shot))
