"""Seeded synthetic inputs for the RTM hot path.

This module is shared by the CUDA path, the FP64 oracle, the tests and the
benchmark. It holds input synthesis only: velocity models, acquisition
geometry, random test directions and the workload descriptions. It contains
none of the method's arithmetic (no stencil, no wavelet, no sponge, no
imaging); each side computes those itself from the numbers produced here.

The paper (Sec. I, Sec. II) names no dataset: it describes an RTM code that
applies a high-order stencil to a 3D block in each time step. Every input here
is a seeded synthetic model with the shapes and value ranges of the workloads
listed in ``WORKLOADS``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "courant_dt",
    "two_layer_velocity",
    "smooth_random_velocity",
    "blob_perturbation",
    "layered_salt_velocity",
    "surface_receivers",
    "batch_apertures",
    "random_directions",
    "standard_normal",
]


def standard_normal(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """N(0,1) samples from numpy's PCG64 bit generator with a fixed seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(size=shape, dtype=dtype)


def courant_dt(dx: float, vmax: float, courant: float = 0.5) -> float:
    """Time step for a 3D Courant number ``courant = vmax*dt*sqrt(3)/dx``.

    The workloads quote "dt at CFL 0.5". Read literally as vmax*dt/dx = 0.5
    the 8th-order leapfrog is unstable (its limit is 0.4529), so the number is
    taken as the 3D Courant number, giving vmax*dt/dx = 0.2887.
    """
    return courant * dx / (vmax * math.sqrt(3.0))


# ----------------------------------------------------------------------------
# velocity models (model grid, C order [z][y][x], metres per second)
# ----------------------------------------------------------------------------

def two_layer_velocity(nx: int, ny: int, nz: int, v_top: float, v_bottom: float,
                       z_interface: int, dtype=np.float64) -> np.ndarray:
    """Two flat layers: ``v_top`` for z < z_interface, ``v_bottom`` below."""
    v = np.full((nz, ny, nx), v_top, dtype=dtype)
    v[z_interface:] = v_bottom
    return v


def _gaussian_weights(sigma: float, truncate: float = 4.0) -> np.ndarray:
    radius = int(truncate * sigma + 0.5)
    x = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-0.5 * (x / sigma) ** 2)
    return w / w.sum()


def _smooth_torch(noise: np.ndarray, sigma: float, device) -> np.ndarray:
    """Separable Gaussian filter on a torch device, symmetric ('reflect'
    in scipy's sense: d c b a | a b c d) boundary handling."""
    import torch
    import torch.nn.functional as F

    w = torch.tensor(_gaussian_weights(sigma), dtype=torch.float32, device=device)
    rad = (w.numel() - 1) // 2
    t = torch.from_numpy(noise).to(device=device, dtype=torch.float32)
    for axis in range(3):
        t = t.movedim(axis, -1).contiguous()
        n = t.shape[-1]
        if rad > n:
            raise ValueError("grid smaller than the Gaussian filter radius")
        left = t[..., :rad].flip(-1)
        right = t[..., n - rad:].flip(-1)
        tp = torch.cat([left, t, right], dim=-1)
        shp = tp.shape
        out = F.conv1d(tp.reshape(-1, 1, shp[-1]), w.view(1, 1, -1))
        t = out.reshape(*shp[:-1], n).movedim(-1, axis)
    return t


def smooth_random_velocity(nx: int, ny: int, nz: int, sigma: float = 8.0,
                           vmin: float = 1500.0, vmax: float = 4500.0,
                           seed: int = 2, device=None, dtype=np.float64):
    """Smooth random velocity: white noise, Gaussian-filtered with ``sigma``
    cells, rescaled so that its minimum is exactly ``vmin`` and its maximum
    exactly ``vmax``.

    With ``device=None`` the filter runs on the CPU (scipy, float64) and a
    numpy array is returned. With a torch device (large grids) it runs there in
    float32 and a float32 torch tensor on that device is returned; the noise is
    the same seeded numpy draw in both cases.
    """
    if device is None:
        from scipy.ndimage import gaussian_filter

        noise = standard_normal((nz, ny, nx), seed, np.float64)
        s = gaussian_filter(noise, sigma, mode="reflect", truncate=4.0)
        lo, hi = s.min(), s.max()
        v = vmin + (vmax - vmin) * (s - lo) / (hi - lo)
        return v.astype(dtype, copy=False)
    noise = standard_normal((nz, ny, nx), seed, np.float32)
    s = _smooth_torch(noise, sigma, device)
    lo, hi = s.min(), s.max()
    v = vmin + (vmax - vmin) * (s - lo) / (hi - lo)
    # pin the extremes exactly despite float32 rounding of the rescale
    v = v.clamp_(vmin, vmax)
    return v


def blob_perturbation(v, amplitude: float = 0.05, radius: float = 16.0,
                      center: Optional[Tuple[float, float, float]] = None):
    """``v * (1 + amplitude * exp(-|x - x_c|^2 / (2 radius^2)))`` with the
    blob centred in the model unless ``center`` (x, y, z) is given. Works on
    numpy arrays and torch tensors."""
    nz, ny, nx = v.shape
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    cx, cy, cz = center
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    r2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
    bump = 1.0 + amplitude * np.exp(-r2 / (2.0 * radius * radius))
    if isinstance(v, np.ndarray):
        return v * bump.astype(v.dtype)
    import torch

    return v * torch.from_numpy(bump.astype(np.float32)).to(v.device)


def thin_bed_reflectors(v, depths=(96, 192, 288), thickness: int = 8,
                       contrast: float = 0.08):
    """``v`` with thin horizontal beds: at each model depth index in
    ``depths`` a bed of ``thickness`` cells whose velocity is scaled by
    ``1 + contrast`` (alternating in sign from bed to bed). Reflections from
    their top and bottom edges make the scattered data that an RTM images.
    Works on numpy arrays and torch tensors."""
    nz = v.shape[0]
    scale = np.ones(nz, dtype=np.float64)
    for i, d in enumerate(depths):
        sign = 1.0 if i % 2 == 0 else -1.0
        scale[max(0, d):min(nz, d + thickness)] = 1.0 + sign * contrast
    if isinstance(v, np.ndarray):
        return v * scale.astype(v.dtype)[:, None, None]
    import torch

    return v * torch.from_numpy(scale.astype(np.float32)).to(v.device)[:, None, None]


def layered_salt_velocity(nx: int, ny: int, nz: int, seed: int = 4,
                          n_layers: int = 5, v_first: float = 1500.0,
                          v_last: float = 4000.0, n_bodies: int = 6,
                          v_salt: float = 4500.0, axis_range=(32, 128),
                          dtype=np.float32) -> np.ndarray:
    """Layered background with salt-like ellipsoids.

    ``n_layers`` layers with velocities linearly spaced from ``v_first`` to
    ``v_last``; the interfaces are gently dipping planes at seeded depths.
    ``n_bodies`` ellipsoids with seeded centres and semi-axes in
    ``axis_range`` cells are set to ``v_salt``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    v = np.empty((nz, ny, nx), dtype=dtype)
    vel = np.linspace(v_first, v_last, n_layers)
    depths = np.sort(rng.uniform(0.1, 0.9, size=n_layers - 1)) * nz
    dips = rng.uniform(-0.05, 0.05, size=(n_layers - 1, 2))
    y = np.arange(ny, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    zc = np.arange(nz, dtype=np.float64)
    layer = np.zeros((nz, ny, nx), dtype=np.int8)
    for i in range(n_layers - 1):
        surf = depths[i] + dips[i, 0] * (x - nx / 2) + dips[i, 1] * (y - ny / 2)
        layer += (zc[:, None, None] >= surf[None]).astype(np.int8)
    v[...] = vel[layer]
    lo, hi = axis_range
    for _ in range(n_bodies):
        c = rng.uniform([0, 0, nz * 0.3], [nx, ny, nz * 0.9])
        a = rng.uniform(lo, hi, size=3)
        z0, z1 = int(max(0, c[2] - a[2])), int(min(nz, c[2] + a[2] + 1))
        y0, y1 = int(max(0, c[1] - a[1])), int(min(ny, c[1] + a[1] + 1))
        x0, x1 = int(max(0, c[0] - a[0])), int(min(nx, c[0] + a[0] + 1))
        if z0 >= z1 or y0 >= y1 or x0 >= x1:
            continue
        zz = ((np.arange(z0, z1) - c[2]) / a[2])[:, None, None] ** 2
        yy = ((np.arange(y0, y1) - c[1]) / a[1])[None, :, None] ** 2
        xx = ((np.arange(x0, x1) - c[0]) / a[0])[None, None, :] ** 2
        inside = (xx + yy + zz) <= 1.0
        sub = v[z0:z1, y0:y1, x0:x1]
        sub[inside] = v_salt
    return v


# ----------------------------------------------------------------------------
# acquisition geometry (model coordinates)
# ----------------------------------------------------------------------------

def surface_receivers(nx: int, ny: int, z: int = 2, stride: int = 1) -> np.ndarray:
    """Receivers at every ``stride``-th (x, y) of the model plane ``z``.

    Returns int32 ``[nrec][3]`` model coordinates (x, y, z), x fastest.
    """
    ys, xs = np.meshgrid(np.arange(0, ny, stride), np.arange(0, nx, stride), indexing="ij")
    rec = np.stack([xs.ravel(), ys.ravel(), np.full(xs.size, z)], axis=1)
    return np.ascontiguousarray(rec.astype(np.int32))


def batch_apertures(nshots: int, model_shape, seed: int = 4,
                    xy_range=(128, 384), z_range=(256, 512), quantum: int = 32):
    """Seeded uneven shot apertures inside a model ``(nz, ny, nx)``.

    Each aperture has sizes drawn uniformly on multiples of ``quantum`` in
    ``xy_range`` (x and y) and ``z_range`` (z), starts at the surface (z = 0)
    and is centred on a seeded surface point, clipped to the model. Returns
    int32 arrays ``origin[nshots][3]`` and ``size[nshots][3]`` in (x, y, z).
    """
    nz, ny, nx = model_shape
    rng = np.random.Generator(np.random.PCG64(seed))
    q = quantum
    sx = rng.integers(xy_range[0] // q, xy_range[1] // q + 1, size=nshots) * q
    sy = rng.integers(xy_range[0] // q, xy_range[1] // q + 1, size=nshots) * q
    sz = rng.integers(z_range[0] // q, z_range[1] // q + 1, size=nshots) * q
    sx = np.minimum(sx, nx)
    sy = np.minimum(sy, ny)
    sz = np.minimum(sz, nz)
    cx = rng.integers(0, nx, size=nshots)
    cy = rng.integers(0, ny, size=nshots)
    ox = np.clip(cx - sx // 2, 0, nx - sx)
    oy = np.clip(cy - sy // 2, 0, ny - sy)
    oz = np.zeros(nshots, dtype=np.int64)
    origin = np.stack([ox, oy, oz], axis=1).astype(np.int32)
    size = np.stack([sx, sy, sz], axis=1).astype(np.int32)
    return origin, size


def random_directions(shape, count: int, seed: int = 7) -> np.ndarray:
    """``count`` seeded N(0,1) fields of ``shape`` (float64), for
    finite-difference gradient checks."""
    return standard_normal((count,) + tuple(shape), seed, np.float64)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Workload:
    """One RTM workload: model grid, discretisation, geometry and storage."""

    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    nb: int
    radius: int
    nt: int
    f0: float
    src: Tuple[int, int, int]
    rec_z: int
    velocity: str            # "two_layer" | "smooth_random" | "layered_salt"
    vmin: float
    vmax: float
    seed: int
    storage: str = "all"     # "all" | "ckpt"
    ckpt_every: int = 0
    image_every: int = 1
    courant: float = 0.5

    @property
    def dt(self) -> float:
        return courant_dt(self.dx, self.vmax, self.courant)

    @property
    def t0(self) -> float:
        return 1.0 / self.f0

    @property
    def padded_shape(self):
        return (self.nz + 2 * self.nb, self.ny + 2 * self.nb, self.nx + 2 * self.nb)

    def velocity_model(self, device=None):
        if self.velocity == "two_layer":
            return two_layer_velocity(self.nx, self.ny, self.nz, self.vmin, self.vmax,
                                      self.nz // 2)
        if self.velocity == "smooth_random":
            return smooth_random_velocity(self.nx, self.ny, self.nz, 8.0, self.vmin,
                                          self.vmax, self.seed, device=device)
        if self.velocity == "layered_salt":
            return layered_salt_velocity(self.nx, self.ny, self.nz, self.seed)
        raise ValueError(self.velocity)

    def receivers(self) -> np.ndarray:
        return surface_receivers(self.nx, self.ny, self.rec_z)

    def scaled(self, **changes) -> "Workload":
        return dataclasses.replace(self, **changes)


WORKLOADS = {
    # plain RTM of one shot on a two-layer model, every source snapshot stored
    "two_layer_64": Workload(
        name="two_layer_64", nx=64, ny=64, nz=64, dx=10.0, nb=20, radius=4, nt=300,
        f0=15.0, src=(32, 32, 4), rec_z=2, velocity="two_layer", vmin=1500.0,
        vmax=2500.0, seed=1, storage="all"),
    # single-shot throughput: 512^3 smooth random model, checkpoint every 50
    "smooth_512": Workload(
        name="smooth_512", nx=512, ny=512, nz=512, dx=10.0, nb=32, radius=4, nt=2000,
        f0=20.0, src=(256, 256, 4), rec_z=2, velocity="smooth_random", vmin=1500.0,
        vmax=4500.0, seed=2, storage="ckpt", ckpt_every=50),
    # velocity gradient of the data misfit: 256^3, checkpoint every 25
    "gradient_256": Workload(
        name="gradient_256", nx=256, ny=256, nz=256, dx=10.0, nb=32, radius=4, nt=1000,
        f0=20.0, src=(128, 128, 4), rec_z=2, velocity="smooth_random", vmin=1500.0,
        vmax=4500.0, seed=3, storage="ckpt", ckpt_every=25),
    # learned snapshot compression: 384^3, imaging every 4 steps
    "learned_384": Workload(
        name="learned_384", nx=384, ny=384, nz=384, dx=10.0, nb=32, radius=4, nt=3000,
        f0=20.0, src=(192, 192, 4), rec_z=2, velocity="smooth_random", vmin=1500.0,
        vmax=4500.0, seed=5, storage="ckpt", ckpt_every=4, image_every=4),
}

# batched shots: 32 apertures of a 1024 x 1024 x 512 layered/salt model,
# 16th-order stencil, 1500 steps each
BATCH_WORKLOAD = dict(model_shape=(512, 1024, 1024), nshots=32, radius=8, nt=1500,
                      f0=20.0, dx=10.0, nb=32, vmax=4500.0, seed=4)


# ----------------------------------------------------------------------------
# seeded initial weights of the snapshot-compression autoencoder
# ----------------------------------------------------------------------------

AE_SHAPES = (("W1", (32, 2, 2, 2), 8, 1.0), ("b1", (32,), 0, 0.0),
             ("W2", (16, 3, 3, 3, 32), 27 * 32, 0.5), ("b2", (16,), 0, 0.0),
             ("W3", (32, 4, 4, 4, 16), 8 * 16, 1.0), ("b3", (32,), 0, 0.0),
             ("W4", (2, 2, 2, 32), 32, 0.5), ("b4", (1,), 0, 0.0))


def ae_init_params(seed: int = 0):
    """Seeded initial autoencoder parameters (He-style: N(0,1) * gain *
    sqrt(2 / fan_in); biases zero), as a dict of float64 arrays in the order
    W1 b1 W2 b2 W3 b3 W4 b4."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for name, shape, fan_in, gain in AE_SHAPES:
        if fan_in:
            out[name] = rng.standard_normal(shape) * math.sqrt(2.0 / fan_in) * gain
        else:
            out[name] = np.zeros(shape)
    return out


def ae_flat(params) -> np.ndarray:
    """Flat float64 vector of autoencoder parameters in the order of AE_SHAPES."""
    return np.concatenate([np.asarray(params[n], np.float64).ravel() for n, *_ in AE_SHAPES])
