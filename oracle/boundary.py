"""Source-wavefield recovery by reverse time stepping from stored boundary
bands -- TEST INFRASTRUCTURE ONLY (imported by ``tests/`` and nothing in the
product).

The imaging condition (Sec. I: the image is formed from the simulated source
and receiver pressure fields) needs the source field at each imaging step, in
reverse time order, while the receiver field is propagated backwards. The
paper does not say how the source field is kept. Besides storing it or
recomputing it from checkpoints it can be run backwards. Inside the model
region the sponge factor is 1, so the forward update

    u^{n+1} = 2 u^n + c L u^n - u^{n-1} + [x = s] c_s w^n / dx^3

can be solved for the older state:

    u^{n-1} = 2 u^n + c L u^n - u^{n+1} + [x = s] c_s w^n / dx^3.

That holds at every cell whose whole star lies in the model region (inner
cells: at least r cells from each of its six faces). The other model cells
(the band) have stencil neighbours in the sponge, where the damped update
cannot be inverted stably, so the forward pass keeps the band of every state
and the reverse pass takes those cells from it. Written out here in FP64 on
whole arrays, with the oracle's own Laplacian.
"""
from __future__ import annotations

from typing import Dict

import numpy as np


def band_mask(model_shape, r: int) -> np.ndarray:
    """Boolean mask of the model cells within ``r`` cells of a model face
    (shape [nz][ny][nx])."""
    nz, ny, nx = model_shape
    m = np.zeros((nz, ny, nx), dtype=bool)
    m[:r] = m[nz - r:] = True
    m[:, :r] = m[:, ny - r:] = True
    m[:, :, :r] = m[:, :, nx - r:] = True
    return m


def reverse_states(grid, w: np.ndarray, src: int, last: np.ndarray,
                   bands: Dict[int, np.ndarray]) -> Dict[int, np.ndarray]:
    """States ``u^m`` on the model region for ``m = nt-2 .. 1``, from the last
    two states ``last = (u^{nt-1}, u^{nt})`` (padded, as the forward run
    leaves them) and the band values ``bands[m] = u^m[band_mask]``.

    ``grid`` is an ``oracle.Grid`` (its sponge must be 1 on the model region),
    ``w`` the wavelet samples, ``src`` the linear padded source index."""
    nb, r = grid.nb, grid.r
    nz, ny, nx = grid.model_shape
    mask = band_mask((nz, ny, nx), r)
    inner = slice(nb, nb + nz), slice(nb, nb + ny), slice(nb, nb + nx)
    g = grid.g()[inner]
    if not np.all(g == 1.0):
        raise ValueError("the sponge reaches into the model region")
    nt = w.shape[0]
    sz, rem = divmod(int(src), grid.NY * grid.NX)
    sy, sx = divmod(rem, grid.NX)
    ms = (sz - nb, sy - nb, sx - nb)
    src_inner = all(r <= ms[i] < (nz, ny, nx)[i] - r for i in range(3))
    inj = grid.c[sz, sy, sx] / grid.dx ** 3

    def model_only(u):  # padded array holding the model region only
        out = np.zeros(grid.shape)
        out[inner] = u[inner]
        return out

    hi = model_only(np.asarray(last[1], dtype=np.float64))  # u^{m+2}
    lo = model_only(np.asarray(last[0], dtype=np.float64))  # u^{m+1}
    states = {}
    for m in range(nt - 2, 0, -1):
        # undo forward step n = m + 1, which made u^{m+2} from u^{m+1} and u^m
        prev = 2.0 * lo + grid.c * grid.laplacian(lo) - hi
        um = prev[inner].copy()
        if src_inner:
            um[ms] += inj * w[m + 1]
        um[mask] = bands[m]
        states[m] = um
        nxt = np.zeros(grid.shape)
        nxt[inner] = um
        hi, lo = lo, nxt
    return states
