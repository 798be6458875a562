"""Off-grid sources and receivers for the FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` use it; the CUDA path never does. The paper's time step
includes "interpolation where necessary" (Sec. II) without saying what is
interpolated. The reading here: a source or receiver may sit between grid
points, and is represented on the grid by Kaiser-windowed sinc weights
(Hicks 2002, "Arbitrary source and receiver positioning in finite-difference
schemes using Kaiser windowed sinc functions"). Along one axis, a point at
position xi (in grid cells, padded coordinates) has the weights

    w_i = sinc(i - xi) * I0(b sqrt(1 - ((i - xi) / R)^2)) / I0(b),   |i - xi| <= R,

on the 2R grid points around it (R = 4, b = 4.14: the Kaiser parameter that
keeps the interpolation error of waves up to 3 cells per wavelength,
k <= 2 pi / 3, smallest for this half-width; Hicks tabulates the same
value). On an axis where xi is a grid point the weights are that single
point. The 3-D weight of a tap is the product of its three axis weights;
taps outside the padded grid are dropped (Dirichlet ghost cells).

With W_t the tap weights of a point:
    source injection   u^{n+1}[t] += c[t] W_t w^n / dx^3
    receiver gather    d[n] = sum_t W_t u^{n+1}[t]
    adjoint injection  mu^m[t] += c[t] g[t] W_t r^{m-1} / dx^3
which reduce to the on-grid forms for a single tap of weight 1, and keep
the receiver propagation the exact transpose of the forward map.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

HALF_WIDTH = 4
KAISER_B = 4.14


def axis_weights(xi: float, n: int, half_width: int = HALF_WIDTH,
                 b: float = KAISER_B) -> Tuple[np.ndarray, np.ndarray]:
    """Grid indices in [0, n) and weights of one axis for position xi."""
    if float(xi) == float(np.floor(xi)):
        i = int(xi)
        return (np.array([i]), np.array([1.0])) if 0 <= i < n else (np.zeros(0, int),
                                                                     np.zeros(0))
    lo = int(np.floor(xi)) - half_width + 1
    idx = np.arange(lo, lo + 2 * half_width)
    d = idx - float(xi)
    win = np.i0(b * np.sqrt(np.clip(1.0 - (d / half_width) ** 2, 0.0, None))) / np.i0(b)
    w = np.sinc(d) * win
    keep = (idx >= 0) & (idx < n)
    return idx[keep], w[keep]


def point_taps(pos_xyz, nb: int, padded_shape) -> Tuple[np.ndarray, np.ndarray]:
    """Linear padded indices and 3-D weights of a point at model coordinates
    (x, y, z) (floats; the padded position is the model one plus nb)."""
    NZ, NY, NX = padded_shape
    ix, wx = axis_weights(pos_xyz[0] + nb, NX)
    iy, wy = axis_weights(pos_xyz[1] + nb, NY)
    iz, wz = axis_weights(pos_xyz[2] + nb, NZ)
    lin = ((iz[:, None, None] * NY + iy[None, :, None]) * NX + ix[None, None, :]).ravel()
    w = (wz[:, None, None] * wy[None, :, None] * wx[None, None, :]).ravel()
    return lin.astype(np.int64), w


def taps_of(points, nb: int, padded_shape) -> List[Tuple[np.ndarray, np.ndarray]]:
    return [point_taps(p, nb, padded_shape) for p in np.asarray(points, np.float64)]


def _flat(taps):
    """All taps of a list of points: indices, weights and owning point."""
    if not len(taps):
        return np.zeros(0, np.int64), np.zeros(0), np.zeros(0, np.int64)
    return (np.concatenate([t[0] for t in taps]), np.concatenate([t[1] for t in taps]),
            np.concatenate([np.full(len(t[0]), j, np.int64) for j, t in enumerate(taps)]))


def forward(grid, w: np.ndarray, src_taps, rec_taps, keep_u: bool = False):
    """Forward modelling from zero fields with a distributed source and
    receivers: each step is the oracle's source-free leapfrog step, then the
    injection at the source taps, then the gather at the receiver taps (the
    order of the on-grid oracle). Returns data [nt][nrec] and, on request,
    the model-region snapshots u [nt] (u^{n+1})."""
    nt = len(w)
    dx3 = grid.dx ** 3
    c = grid.c.ravel()
    u_prev = np.zeros(grid.shape)
    u_cur = np.zeros(grid.shape)
    data = np.zeros((nt, len(rec_taps)))
    nb = grid.nb
    snaps = np.zeros((nt,) + grid.model_shape) if keep_u else None
    s_idx, s_w = src_taps
    r_idx, r_w, r_own = _flat(rec_taps)
    for n in range(nt):
        u_next = grid.step(u_cur, u_prev)
        flat = u_next.reshape(-1)
        flat[s_idx] += c[s_idx] * s_w * w[n] / dx3
        if len(rec_taps):
            data[n] = np.bincount(r_own, weights=r_w * flat[r_idx], minlength=len(rec_taps))
        if keep_u:
            snaps[n] = u_next[nb:grid.NZ - nb, nb:grid.NY - nb, nb:grid.NX - nb]
        u_prev, u_cur = u_cur, u_next
    return {"data": data, "u": snaps, "last": (u_prev, u_cur)}


def adjoint(grid, rec_taps, resid: np.ndarray, snap_u=None, image_every: int = 1,
            src_taps=None):
    """Receiver propagation backward in time with the data injected at the
    receiver taps, and the zero-lag image sum over m % image_every == 0 of
    u^m mu^m over the model region (snap_u[m - 1] = u^m). With the source
    taps, also the trace at the source, src_adj[m - 1] = sum_t W_t mu^m[t] /
    g[t]: the transpose of the source injection in the scaled adjoint."""
    nt = resid.shape[0]
    dx3 = grid.dx ** 3
    c = grid.c.ravel()
    g = grid.g().ravel()
    idx_all, w_all, owner = _flat(rec_taps)
    coef = c[idx_all] * g[idx_all] * w_all / dx3
    N = c.size
    nb = grid.nb
    mu2 = np.zeros(grid.shape)
    mu1 = np.zeros(grid.shape)
    image = np.zeros(grid.model_shape) if snap_u is not None else None
    src_adj = np.zeros(nt)
    for m in range(nt, 0, -1):
        mu0 = grid.step(mu1, mu2)
        flat = mu0.reshape(-1)
        if len(idx_all):
            flat += np.bincount(idx_all, weights=coef * resid[m - 1, owner], minlength=N)
        if image is not None and m % image_every == 0:
            image += snap_u[m - 1] * mu0[nb:grid.NZ - nb, nb:grid.NY - nb, nb:grid.NX - nb]
        if src_taps is not None:
            s_idx, s_w = src_taps
            src_adj[m - 1] = float(np.sum(s_w * flat[s_idx] / g[s_idx]))
        mu2, mu1 = mu1, mu0
    return {"image": image, "src_adj": src_adj, "last": (mu2, mu1)}
