"""Snapshot-compression autoencoder: binding of the codec entry points of
librtm (tensor-core encode, decode, training step, GEMM engine check).

A float32 snapshot (any strided [nz][ny][nx] view with x contiguous, every
side a multiple of 4) becomes a bfloat16 latent [nz/4][ny/4][nx/4][16] plus
one float32 scale: 8x fewer bytes. Parameters are one float32 vector of
``NPARAMS`` values in the order W1 b1 W2 b2 W3 b3 W4 b4.
"""
from __future__ import annotations

import ctypes

import torch

from ._lib import call, lib

NPARAMS = 47185


def _p(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must be %s" % (name, dtype))
    return ctypes.c_void_p(t.data_ptr())


def _s(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def workspace_size(nx: int, ny: int, nz: int) -> int:
    n = lib().rtm_ae_workspace_size(nx, ny, nz)
    if n == 0:
        raise ValueError("codec volume %dx%dx%d: sides must be multiples of 4" % (nx, ny, nz))
    return int(n)


def alloc_workspace(shape, device="cuda") -> torch.Tensor:
    nz, ny, nx = shape
    return torch.empty(workspace_size(nx, ny, nz), dtype=torch.uint8, device=device)


def _vol(t: torch.Tensor):
    if t.dim() != 3 or t.stride(2) != 1 or t.dtype != torch.float32:
        raise ValueError("snapshot must be a float32 [nz][ny][nx] view with x contiguous")
    nz, ny, nx = t.shape
    return t.stride(1), t.stride(0), nx, ny, nz


def latent_shape(shape):
    nz, ny, nx = shape
    return (nz // 4, ny // 4, nx // 4, 16)


def encode(params: torch.Tensor, snap: torch.Tensor, ws: torch.Tensor, latent=None, scale=None,
           stream=None):
    sy, sz, nx, ny, nz = _vol(snap)
    if latent is None:
        latent = torch.empty(latent_shape(snap.shape), dtype=torch.bfloat16, device=snap.device)
    if scale is None:
        scale = torch.empty(1, dtype=torch.float32, device=snap.device)
    call("rtm_ae_encode", _p(params, torch.float32, "params"), _p(snap), ctypes.c_int64(sy),
         ctypes.c_int64(sz), nx, ny, nz, _p(latent, torch.bfloat16, "latent"),
         _p(scale, torch.float32, "scale"), _p(ws), ctypes.c_size_t(ws.numel()), _s(stream))
    return latent, scale


def decode(params: torch.Tensor, latent: torch.Tensor, scale, ws: torch.Tensor, out=None,
           shape=None, stream=None):
    if out is None:
        nz4, ny4, nx4, _ = latent.shape
        out = torch.empty((4 * nz4, 4 * ny4, 4 * nx4), dtype=torch.float32, device=latent.device)
    sy, sz, nx, ny, nz = _vol(out)
    call("rtm_ae_decode", _p(params, torch.float32, "params"), _p(latent, torch.bfloat16, "latent"),
         _p(scale, torch.float32, "scale"), _p(out), ctypes.c_int64(sy), ctypes.c_int64(sz), nx,
         ny, nz, _p(ws), ctypes.c_size_t(ws.numel()), _s(stream))
    return out


def train_step(params, adam_m, adam_v, step: int, lr: float, batch: torch.Tensor,
               ws: torch.Tensor, grad_out=None, loss=None, stream=None):
    """One Adam step on a batch [B][nz][ny][nx] of snapshots (lr = 0: only the
    loss and the gradient). Returns the mean loss (float64 device scalar)."""
    if batch.dim() != 4 or not batch.is_contiguous():
        raise ValueError("batch must be a contiguous [B][nz][ny][nx] tensor")
    B, nz, ny, nx = batch.shape
    if loss is None:
        loss = torch.empty(1, dtype=torch.float64, device=batch.device)
    call("rtm_ae_train_step", _p(params, torch.float32, "params"), _p(adam_m), _p(adam_v),
         int(step), ctypes.c_float(lr), _p(batch, torch.float32, "batch"), int(B), nx, ny, nz,
         _p(loss, torch.float64, "loss"), _p(grad_out), _p(ws), ctypes.c_size_t(ws.numel()),
         _s(stream))
    return loss


def gemm_bf16(A: torch.Tensor, B: torch.Tensor, status=None, stream=None) -> torch.Tensor:
    """C[M][N] = A[M][K] B[N][K]^T on the tcgen05 engine (bf16 in, f32 out)."""
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    call("rtm_ae_gemm_bf16", _p(A.contiguous(), torch.bfloat16, "A"),
         _p(B.contiguous(), torch.bfloat16, "B"), _p(C), M, K, N,
         _p(status, torch.int32, "status"), _s(stream))
    return C


def set_decoder(which: str = "auto") -> None:
    """Inference decoder: "auto", "gemm" (GEMM-engine decoder) or "march"
    (z-marching kernel with TMA plane loads read in place by the tensor
    cores). Both give the same values."""
    code = {"auto": 0, "gemm": 1, "march": 2}[which]
    call("rtm_ae_set_decoder", code)


def set_encoder(which: str = "auto") -> None:
    """Inference encoder: "auto", "gemm" (GEMM-engine encoder) or "march"
    (z-marching kernel: h1 kept in shared memory, E1 and E2 on the tensor
    cores). Both give the same values."""
    code = {"auto": 0, "gemm": 1, "march": 2}[which]
    call("rtm_ae_set_encoder", code)


def _time_codec(n: int, reps: int = 10, seed: int = 0):
    """Encode and decode of a random n^3 snapshot; returns (encode ms, decode ms)."""
    import numpy as np

    import rtm_inputs

    P = torch.from_numpy(rtm_inputs.ae_flat(rtm_inputs.ae_init_params(seed)).astype(np.float32))
    P = P.cuda()
    s = torch.randn(n, n, n, device="cuda")
    ws = alloc_workspace((n, n, n))
    lat, sc = encode(P, s, ws)
    r = decode(P, lat, sc, ws)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    for _ in range(reps):
        encode(P, s, ws, latent=lat, scale=sc)
    e[1].record()
    for _ in range(reps):
        decode(P, lat, sc, ws, out=r)
    e[2].record()
    torch.cuda.synchronize()
    return e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps


if __name__ == "__main__":
    import sys

    n = int(sys.argv[1]) if len(sys.argv) > 1 else 384
    reps = int(sys.argv[2]) if len(sys.argv) > 2 else 10
    enc, dec = _time_codec(n, reps)
    print("codec %d^3: encode %.3f ms, decode %.3f ms" % (n, enc, dec))
