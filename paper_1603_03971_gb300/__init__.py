"""GB300-native RTM hot path: Python binding of librtm.

Every numerical step runs in the library's CUDA kernels (``csrc/``); this
module only marshals torch tensors (device memory) and CUDA streams into the C
ABI declared in ``include/rtm.h``. If the library is missing, calls raise.

The method is reverse time migration as the paper describes it (Sec. I): a
wave-propagation solver that applies a high-order stencil to a 3D block of
data in each time step (Sec. II), run forward from the source and backward
from the recorded data, with the two wavefields correlated into an image.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import torch

from ._lib import (RTM_STORE_ALL, RTM_STORE_BOUNDARY, RTM_STORE_CKPT, RTM_STORE_DECIMATED,
                   RTM_STORE_LEARNED, RTM_STORE_REVOLVE, RTM_VEL_V, RTM_VEL_V2,
                   RtmError, RtmParams, RtmStats, call, lib)

__all__ = [
    "RtmParams", "RtmError", "make_params", "params_for", "padded_shape", "workspace_size",
    "host_workspace_size", "alloc_workspace", "model_prep", "forward", "backward_image",
    "shot", "grad", "misfit", "check", "shot_host", "forward_learned",
    "backward_image_learned", "shot_learned", "snapshot", "set_tuning", "set_timing", "stats",
    "reset_stats", "RtmMisfit", "version", "decomp_plan", "decomp_workspace_size",
    "forward_decomposed", "offgrid_taps", "forward_offgrid", "shot_offgrid",
]


def version() -> str:
    return lib().rtm_version().decode()


def make_params(nx, ny, nz, nb, radius, nt, dx, dt, f0, t0, src, nrec, storage="all",
                ckpt_every=0, image_every=1, want_grad=False) -> RtmParams:
    p = RtmParams()
    p.nx, p.ny, p.nz, p.nb, p.radius, p.nt = nx, ny, nz, nb, radius, nt
    p.dx, p.dt, p.f0, p.t0 = float(dx), float(dt), float(f0), float(t0)
    p.src_x, p.src_y, p.src_z = (int(v) for v in src)
    p.nrec = int(nrec)
    p.storage = {"all": RTM_STORE_ALL, "ckpt": RTM_STORE_CKPT,
                 "learned": RTM_STORE_LEARNED, "revolve": RTM_STORE_REVOLVE,
                 "boundary": RTM_STORE_BOUNDARY, "decimated": RTM_STORE_DECIMATED}[storage]
    p.ckpt_every = int(ckpt_every)
    p.image_every = int(image_every)
    p.want_grad = 1 if want_grad else 0
    return p


def params_for(w, nrec: Optional[int] = None, **changes) -> RtmParams:
    """Parameters of an ``rtm_inputs.Workload`` (receivers: its surface plane)."""
    if nrec is None:
        nrec = w.nx * w.ny
    kw = dict(nx=w.nx, ny=w.ny, nz=w.nz, nb=w.nb, radius=w.radius, nt=w.nt, dx=w.dx,
              dt=w.dt, f0=w.f0, t0=w.t0, src=w.src, nrec=nrec, storage=w.storage,
              ckpt_every=w.ckpt_every, image_every=w.image_every)
    kw.update(changes)
    return make_params(**kw)


def padded_shape(p: RtmParams):
    return (p.nz + 2 * p.nb, p.ny + 2 * p.nb, p.nx + 2 * p.nb)


def model_shape(p: RtmParams):
    return (p.nz, p.ny, p.nx)


def workspace_size(p: RtmParams) -> int:
    n = lib().rtm_workspace_size(ctypes.byref(p))
    if n == 0:
        call("rtm_validate", ctypes.byref(p))
    return int(n)


def host_workspace_size(p: RtmParams) -> int:
    n = lib().rtm_host_workspace_size(ctypes.byref(p))
    if n == 0:
        call("rtm_validate", ctypes.byref(p))
    return int(n)


def alloc_workspace(p: RtmParams, device="cuda", host_io: bool = False) -> torch.Tensor:
    n = host_workspace_size(p) if host_io else workspace_size(p)
    ws = torch.empty(n, dtype=torch.uint8, device=device)
    assert ws.data_ptr() % 256 == 0
    return ws


def _dev(t: Optional[torch.Tensor], dtype=torch.float32, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _host(t: torch.Tensor, dtype, name):
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError("%s must be a contiguous host %s tensor" % (name, dtype))
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ws(ws: torch.Tensor):
    if not ws.is_cuda or ws.dtype != torch.uint8:
        raise ValueError("workspace must be a CUDA uint8 tensor")
    return ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel())


def model_prep(p: RtmParams, vel: torch.Tensor, ws: torch.Tensor, kind: str = "v",
               out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Padded ``c = v^2 dt^2`` from a model-grid velocity (``kind='v'``) or
    squared velocity (``kind='v2'``). Synchronises to check the CFL limit."""
    if out is None:
        out = torch.empty(padded_shape(p), dtype=torch.float32, device=vel.device)
    w, wb = _ws(ws)
    call("rtm_model_prep", ctypes.byref(p), _dev(vel, name="vel"),
         RTM_VEL_V if kind == "v" else RTM_VEL_V2, _dev(out, name="c"), w, wb, _stream(stream))
    return out


def forward(p: RtmParams, c, rec, ws, data=None, u_last=None, stream=None):
    w, wb = _ws(ws)
    call("rtm_forward", ctypes.byref(p), _dev(c, name="c"), _dev(rec, torch.int32, "rec"),
         _dev(data, name="data"), w, wb, _dev(u_last, name="u_last"), _stream(stream))
    return data


def backward_image(p: RtmParams, c, rec, rdata, ws, image, src_adj=None, stream=None):
    w, wb = _ws(ws)
    call("rtm_backward_image", ctypes.byref(p), _dev(c, name="c"),
         _dev(rec, torch.int32, "rec"), _dev(rdata, name="rdata"), w, wb,
         _dev(image, name="image"), _dev(src_adj, name="src_adj"), _stream(stream))
    return image


def shot(p: RtmParams, c, rec, dobs, ws, image, data=None, stream=None):
    w, wb = _ws(ws)
    call("rtm_shot", ctypes.byref(p), _dev(c, name="c"), _dev(rec, torch.int32, "rec"),
         _dev(dobs, name="dobs"), _dev(data, name="data"), w, wb, _dev(image, name="image"),
         _stream(stream))
    return image


def forward_learned(p: RtmParams, c, rec, ae_params, ws, data=None, stream=None):
    w, wb = _ws(ws)
    call("rtm_forward_learned", ctypes.byref(p), _dev(c, name="c"), _dev(rec, torch.int32, "rec"),
         _dev(data, name="data"), _dev(ae_params, name="ae_params"), w, wb, _stream(stream))
    return data


def backward_image_learned(p: RtmParams, c, rec, rdata, ae_params, ws, image, stream=None):
    w, wb = _ws(ws)
    call("rtm_backward_image_learned", ctypes.byref(p), _dev(c, name="c"),
         _dev(rec, torch.int32, "rec"), _dev(rdata, name="rdata"),
         _dev(ae_params, name="ae_params"), w, wb, _dev(image, name="image"), _stream(stream))
    return image


def shot_learned(p: RtmParams, c, rec, dobs, ae_params, ws, image, stream=None):
    w, wb = _ws(ws)
    call("rtm_shot_learned", ctypes.byref(p), _dev(c, name="c"), _dev(rec, torch.int32, "rec"),
         _dev(dobs, name="dobs"), _dev(ae_params, name="ae_params"), w, wb,
         _dev(image, name="image"), _stream(stream))
    return image


def backward_image_illum(p: RtmParams, c, rec, rdata, ws, image, illum, ae_params=None,
                         stream=None):
    """Receiver propagation with the zero-lag image (added to ``image``) and
    the source illumination ``sum_m (u^m)^2`` over the imaging steps (added to
    ``illum``, model grid). Learned storage needs ``ae_params``."""
    w, wb = _ws(ws)
    call("rtm_backward_image_illum", ctypes.byref(p), _dev(c, name="c"),
         _dev(rec, torch.int32, "rec"), _dev(rdata, name="rdata"),
         _dev(ae_params, name="ae_params"), w, wb, _dev(image, name="image"),
         _dev(illum, name="illum"), _stream(stream))
    return image, illum


def image_filter(p: RtmParams, image, ws, illum=None, eps_rel: float = 1e-3,
                 normalized=True, laplacian=True, stream=None):
    """Illumination-normalised image ``I / (illum + eps_rel max illum)`` and/or
    Laplacian-filtered image ``-L I`` (model grid). Returns (normalised or
    None, laplacian or None)."""
    w, wb = _ws(ws)
    norm = torch.empty_like(image) if normalized else None
    lap = torch.empty_like(image) if laplacian else None
    call("rtm_image_filter", ctypes.byref(p), _dev(image, name="image"),
         _dev(illum, name="illum"), ctypes.c_float(eps_rel), _dev(norm, name="normalized"),
         _dev(lap, name="laplacian"), w, wb, _stream(stream))
    return norm, lap


def snapshot(p: RtmParams, ws, m: int, out=None, stream=None):
    """Stored imaging snapshot u^m of a store-all workspace (model grid)."""
    if out is None:
        out = torch.empty(model_shape(p), dtype=torch.float32, device=ws.device)
    w, wb = _ws(ws)
    call("rtm_snapshot", ctypes.byref(p), w, wb, int(m), _dev(out, name="out"), _stream(stream))
    return out


def grad(p: RtmParams, c, rec, resid, ws, out=None, stream=None):
    if out is None:
        out = torch.empty(model_shape(p), dtype=torch.float32, device=c.device)
    w, wb = _ws(ws)
    call("rtm_grad", ctypes.byref(p), _dev(c, name="c"), _dev(rec, torch.int32, "rec"),
         _dev(resid, name="resid"), w, wb, _dev(out, name="grad"), _stream(stream))
    return out


def misfit(d, obs, resid=None, J=None, stream=None):
    if J is None:
        J = torch.empty(1, dtype=torch.float64, device=d.device)
    if d.numel() != obs.numel():
        raise ValueError("data and observed data differ in size")
    call("rtm_misfit", _dev(d, name="d"), _dev(obs, name="obs"), ctypes.c_int64(d.numel()),
         _dev(resid, name="resid"), _dev(J, torch.float64, "J"), _stream(stream))
    return J, resid


TAP_BYTES = 128  # sizeof(rtm_point_taps)


def offgrid_taps(p: RtmParams, src_xyz, rec_xyz, device=None) -> torch.Tensor:
    """Tap tables (Kaiser-windowed sinc weights) of a source and receivers at
    fractional model coordinates (x, y, z), computed by the library on the
    host: a uint8 tensor of (1 + nrec) x 128 bytes (entry 0 the source), on
    ``device`` if given."""
    import numpy as np

    src = np.ascontiguousarray(src_xyz, dtype=np.float64).reshape(3)
    rec = np.ascontiguousarray(rec_xyz, dtype=np.float64).reshape(-1, 3)
    n = 1 + rec.shape[0]
    out = np.zeros(n * TAP_BYTES, dtype=np.uint8)
    got = lib().rtm_offgrid_taps(ctypes.byref(p), src.ctypes.data_as(ctypes.c_void_p),
                                 rec.shape[0], rec.ctypes.data_as(ctypes.c_void_p),
                                 out.ctypes.data_as(ctypes.c_void_p), n)
    if got != n:
        raise RtmError(1, "rtm_offgrid_taps", (lib().rtm_last_error() or b"").decode())
    t = torch.from_numpy(out)
    return t.to(device) if device is not None else t


def _taps(t: torch.Tensor, p: RtmParams):
    if not t.is_cuda or t.dtype != torch.uint8 or t.numel() != (1 + p.nrec) * TAP_BYTES:
        raise ValueError("tap table must be a CUDA uint8 tensor of (1 + nrec) x 128 bytes")
    return ctypes.c_void_p(t.data_ptr())


def forward_offgrid(p: RtmParams, c, taps, ws, data=None, u_last=None, stream=None):
    """Forward modelling with the off-grid source and receivers of a tap table."""
    w, wb = _ws(ws)
    call("rtm_forward_offgrid", ctypes.byref(p), _dev(c, name="c"), _taps(taps, p),
         _dev(data, name="data"), w, wb, _dev(u_last, name="u_last"), _stream(stream))
    return data, u_last


def shot_offgrid(p: RtmParams, c, taps, dobs, ws, image, data=None, stream=None):
    """RTM shot (image +=) with the off-grid source and receivers of a tap table."""
    w, wb = _ws(ws)
    call("rtm_shot_offgrid", ctypes.byref(p), _dev(c, name="c"), _taps(taps, p),
         _dev(dobs, name="dobs"), _dev(data, name="data"), w, wb, _dev(image, name="image"),
         _stream(stream))
    return image


def decomp_plan(p: RtmParams, px: int, py: int):
    """The X-Y decomposition of the padded grid into px x py subdomains (host
    only): one row per subdomain (index j * px + i) of owned padded ranges
    x0, x1, y0, y1 and the neighbours across the W, E, S, N faces (-1 at the
    grid's outer faces)."""
    import numpy as np

    n = px * py
    out = np.zeros((max(n, 1), 8), dtype=np.int32)
    got = lib().rtm_decomp_plan(ctypes.byref(p), int(px), int(py),
                                out.ctypes.data_as(ctypes.c_void_p), n)
    if got < 0:
        raise RtmError(1, "rtm_decomp_plan", (lib().rtm_last_error() or b"").decode())
    return out[:n]


def decomp_workspace_size(p: RtmParams, px: int, py: int) -> int:
    n = lib().rtm_decomp_workspace_size(ctypes.byref(p), int(px), int(py))
    if n == 0:
        raise RtmError(1, "rtm_decomp_workspace_size", (lib().rtm_last_error() or b"").decode())
    return int(n)


def forward_decomposed(p: RtmParams, px: int, py: int, c, rec, ws, data=None, u_last=None,
                       stream=None):
    """Forward modelling on a px x py X-Y decomposition with the halo exchange
    overlapped with the interior stencil (one GPU); same outputs as
    ``forward``."""
    w, wb = _ws(ws)
    call("rtm_forward_decomposed", ctypes.byref(p), int(px), int(py), _dev(c, name="c"),
         _dev(rec, torch.int32, "rec"), _dev(data, name="data"), w, wb,
         _dev(u_last, name="u_last"), _stream(stream))
    return data, u_last


def check(ws, stream=None):
    """Synchronise and raise if a device-side check flagged an error."""
    w, wb = _ws(ws)
    call("rtm_check", w, wb, _stream(stream))


def shot_host(p: RtmParams, vel, rec, dobs, image, ws, kind="v", stream=None):
    """End-to-end shot from host tensors (pinned for asynchronous copies)."""
    w, wb = _ws(ws)
    call("rtm_shot_host", ctypes.byref(p), _host(vel, torch.float32, "vel"),
         RTM_VEL_V if kind == "v" else RTM_VEL_V2, _host(rec, torch.int32, "rec"),
         _host(dobs, torch.float32, "dobs"), _host(image, torch.float32, "image"), w, wb,
         _stream(stream))
    return image


def revolve_cost(nstates: int, slots: int) -> int:
    """Fewest forward steps (in image_every units) of binomial checkpointing
    with ``slots`` checkpoint slots over ``nstates`` imaging steps."""
    return int(lib().rtm_revolve_cost(int(nstates), int(slots)))


def revolve_schedule(nstates: int, slots: int):
    """The binomial checkpointing actions as a list of (op, a, b, c)."""
    n = int(lib().rtm_revolve_schedule(int(nstates), int(slots), None, 0))
    if n < 0:
        raise ValueError("schedule over the planning limit")
    buf = (ctypes.c_int32 * (4 * max(n, 1)))()
    lib().rtm_revolve_schedule(int(nstates), int(slots), ctypes.cast(buf, ctypes.c_void_p), n)
    return [tuple(buf[4 * i:4 * i + 4]) for i in range(n)]


def set_tuning(radius: int, zchunk: int = 0, variant: int = 0):
    call("rtm_set_tuning", radius, zchunk, variant)


MODE_SLOTS = {"fwd": 0, "fwd_snap": 1, "bwd_image": 2, "fwd_lu": 3, "bwd_grad": 4, "rev": 6}


def set_tuning_mode(radius: int, mode: str, zchunk: int):
    """Slab height of one stencil mode (a key of ``MODE_SLOTS``); cleared by
    ``set_tuning``."""
    call("rtm_set_tuning_mode", radius, MODE_SLOTS[mode], zchunk)


STALL_STENCIL, STALL_ENCODER = 0, 1


def set_test_stall(kernel: int, plane: int):
    """Arm (plane >= 0) or disarm (-1) a one-shot wait failure in the next
    launch of the TMA stencil (``STALL_STENCIL``) or the codec encoder
    (``STALL_ENCODER``): the call then reports RTM_ERR_TIMEOUT (testing)."""
    call("rtm_set_test_stall", kernel, plane)


def set_timing(enable: bool):
    call("rtm_set_timing", 1 if enable else 0)


def stats() -> dict:
    s = RtmStats()
    call("rtm_stats_get", ctypes.byref(s))
    names = ["fwd", "fwd_snap", "bwd_image", "fwd_lu", "bwd_grad", "batch", "rev"]
    return {
        "launches": int(s.launches),
        "stencil": {n: {"launches": int(s.stencil_launches[i]), "ms": float(s.stencil_ms[i]),
                        "bytes": float(s.stencil_bytes[i])} for i, n in enumerate(names)},
    }


def reset_stats():
    call("rtm_stats_reset")


class RtmMisfit(torch.autograd.Function):
    """``J(v^2) = 1/2 ||F(v^2) - d_obs||^2`` with its gradient from the
    hand-written adjoint (``rtm_grad``): the forward pass models the data and
    keeps checkpoints (or snapshots) in ``ws``; the backward pass propagates
    the residual backward in time and correlates it with ``L u``.

    ``p`` must have ``want_grad = 1``; ``v2`` is the model-grid squared
    velocity (float32, CUDA). Returns J as a float64 scalar tensor.
    """

    @staticmethod
    def forward(ctx, v2, p: RtmParams, rec, d_obs, ws):
        if not p.want_grad:
            raise ValueError("RtmMisfit needs params with want_grad = 1")
        c = model_prep(p, v2.detach().contiguous(), ws, kind="v2")
        data = torch.empty((p.nt, p.nrec), dtype=torch.float32, device=v2.device)
        forward(p, c, rec, ws, data=data)
        resid = torch.empty_like(data)
        J, _ = misfit(data, d_obs, resid=resid)
        ctx.p, ctx.rec, ctx.ws = p, rec, ws
        ctx.save_for_backward(c, resid)
        return J[0]

    @staticmethod
    def backward(ctx, gJ):
        c, resid = ctx.saved_tensors
        g = grad(ctx.p, c, ctx.rec, resid, ctx.ws)
        return g * gJ.to(g.dtype), None, None, None, None
