"""Imaging-condition variants of the zero-lag RTM image -- TEST
INFRASTRUCTURE ONLY (imported by ``tests/`` and nothing in the product).

The paper images by cross-correlating the source and receiver wavefields
(Sec. I: RTM forms the image from simulated pressure waves) and says nothing
about the image's post-processing. The two standard companions of the
zero-lag condition are written out here in FP64, plainly:

* source illumination ``Lambda(x) = sum_m u^m(x)^2`` over the same imaging
  steps m as the image (the zero-lag autocorrelation of the source
  wavefield), and the illumination-normalised image
  ``I(x) / (Lambda(x) + eps * max_x Lambda)``, which divides out the
  geometric spreading of the source field (eps keeps the quotient bounded
  where the source field never reached);
* the Laplacian-filtered image ``-L I``, with L the 2r-order star Laplacian of
  the propagator (same weights, divided by dx^2) on the model grid and zero
  outside it, which suppresses the smooth low-wavenumber backscatter that
  zero-lag correlation builds up along strong velocity contrasts.
"""
from __future__ import annotations

import numpy as np

from . import coefficients


def illumination(snap_u: np.ndarray, image_every: int = 1) -> np.ndarray:
    """``Lambda = sum_{m = k, 2k, ...} (u^m)^2`` from the model-region
    snapshots ``snap_u[m - 1] = u^m`` (shape [nt][nz][ny][nx])."""
    if image_every < 1:
        raise ValueError("image_every must be >= 1")
    snap_u = np.asarray(snap_u, dtype=np.float64)
    nt = snap_u.shape[0]
    lam = np.zeros(snap_u.shape[1:])
    for m in range(image_every, nt + 1, image_every):
        lam += snap_u[m - 1] * snap_u[m - 1]
    return lam


def normalized_image(image: np.ndarray, illum: np.ndarray, eps_rel: float) -> np.ndarray:
    """``I / (Lambda + eps_rel * max(Lambda))`` (eps_rel > 0)."""
    if not eps_rel > 0:
        raise ValueError("eps_rel must be positive")
    image = np.asarray(image, dtype=np.float64)
    illum = np.asarray(illum, dtype=np.float64)
    return image / (illum + eps_rel * float(illum.max()))


def laplacian_filter(image: np.ndarray, r: int, dx: float) -> np.ndarray:
    """``-L I`` on the model grid: per axis ``a_0 I + sum_k a_k (I[+k] + I[-k])``
    with I = 0 outside the grid, summed over the three axes, divided by
    ``dx^2`` and negated."""
    a = coefficients(r)
    img = np.asarray(image, dtype=np.float64)
    out = np.zeros_like(img)
    for axis in range(3):
        n = img.shape[axis]
        acc = a[0] * img
        for k in range(1, r + 1):
            if k >= n:
                continue
            plus = np.zeros_like(img)
            minus = np.zeros_like(img)
            sl_dst = [slice(None)] * 3
            sl_src = [slice(None)] * 3
            # I[i + k] lands on i (zero where i + k is outside)
            sl_dst[axis], sl_src[axis] = slice(0, n - k), slice(k, n)
            plus[tuple(sl_dst)] = img[tuple(sl_src)]
            # I[i - k] lands on i
            sl_dst[axis], sl_src[axis] = slice(k, n), slice(0, n - k)
            minus[tuple(sl_dst)] = img[tuple(sl_src)]
            acc = acc + a[k] * (plus + minus)
        out += acc
    return -out / (dx * dx)
