"""FP64 CPU oracle for the RTM hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package. The CUDA library never calls it; the two
share no code. Each function cites the part of the method it follows.

The paper (Sec. I) defines RTM as imaging the subsurface by simulating the
propagation of pressure waves, and (Sec. II) its solver as one that applies a
high-order stencil to a 3D block of data in each time step. It gives no
formula. The discrete method written out here is the reading used throughout
this repository:

* 2r-order central second-derivative weights (exact rationals, solved here
  from the moment equations), star Laplacian with zero ghost cells;
* second-order leapfrog in time with a Cerjan-type multiplicative sponge
  ``u^{n+1} = g (2u^n + c L u^n) - g^2 u^{n-1}``, ``c = v^2 dt^2``;
* Ricker source ``w(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2)``
  injected as ``u^{n+1}[s] += c[s] w(n dt) / dx^3``;
* receivers ``d[n][j] = u^{n+1}[rec_j]``;
* receiver propagation: the same recursion backward in time on ``mu`` with the
  data injected as ``mu^m[rec] += c g r^{m-1} / dx^3``; this is the exact
  transpose of the forward map in the scaled variable ``mu = C G lambda / dx^3``;
* zero-lag imaging ``I(x) = sum_m u^m(x) mu^m(x)`` over the model region;
* gradient ``dJ/dc_i = dx^3 / c_i * sum_n mu^{n+1}_i [(L u^n)_i + [i = s] w^n / (dx^3 g_s)]``
  of ``J = 1/2 ||d - d_obs||^2``, folded back onto the model grid through the
  edge padding and multiplied by ``dt^2`` for the gradient with respect to v^2.

Every function here is pinned by the ``-m "not gpu"`` tests against closed
forms, exactness on polynomials, the discrete dispersion relation, the
constant-velocity Green's function, the adjoint dot-product identity, the
imaging identity and central finite differences.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from fractions import Fraction
from typing import Dict, List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liborc.so")
_SRC = os.path.join(_HERE, "rtm_oracle.c")

_lib = None


def build(force: bool = False) -> str:
    """Compile the C core with gcc (OpenMP) into ``oracle/_build/liborc.so``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(ctypes.Structure):
    _fields_ = [
        ("NX", ctypes.c_int), ("NY", ctypes.c_int), ("NZ", ctypes.c_int),
        ("nb", ctypes.c_int), ("r", ctypes.c_int), ("dx", ctypes.c_double),
        ("a", ctypes.c_void_p), ("c", ctypes.c_void_p),
        ("gx", ctypes.c_void_p), ("gy", ctypes.c_void_p), ("gz", ctypes.c_void_p),
    ]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        gp = ctypes.POINTER(_Grid)
        lib.orc_laplacian.argtypes = [gp, vp, vp]
        lib.orc_step.argtypes = [gp, vp, vp, vp]
        lib.orc_forward.argtypes = [gp, ci, vp, i64, ci, vp, vp, vp, vp, vp]
        lib.orc_forward.restype = ci
        lib.orc_adjoint.argtypes = [gp, ci, vp, i64, ci, vp, vp, vp, ci, vp, vp, vp, vp, vp]
        lib.orc_adjoint.restype = ci
        lib.orc_num_threads.restype = ci
        _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the oracle's loops use."""
    return int(_load().orc_num_threads())


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# ----------------------------------------------------------------------------
# stencil weights and the quantities derived from them
# ----------------------------------------------------------------------------

def stencil_coefficients(r: int) -> List[Fraction]:
    """Weights ``a_0..a_r`` of the 2r-order central second derivative.

    The symmetric stencil ``sum_{k=-r..r} a_|k| f(x + k h) / h^2`` matches
    ``f''`` on every polynomial of degree <= 2r+1 iff its even moments satisfy
    ``sum_k a_|k| k^(2m) = 2 delta_{m,1}`` for m = 0..r. The r equations for
    m = 1..r are solved here exactly over the rationals by Gaussian
    elimination, and ``a_0 = -2 sum a_k`` comes from m = 0.
    """
    if r < 1:
        raise ValueError("radius must be >= 1")
    # rows m = 1..r, unknowns a_1..a_r: sum_k a_k k^(2m) = [m == 1]
    A = [[Fraction(k ** (2 * m)) for k in range(1, r + 1)] for m in range(1, r + 1)]
    b = [Fraction(1 if m == 1 else 0) for m in range(1, r + 1)]
    n = r
    for col in range(n):
        piv = next(i for i in range(col, n) if A[i][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        for i in range(n):
            if i != col and A[i][col] != 0:
                f = A[i][col] / A[col][col]
                A[i] = [A[i][j] - f * A[col][j] for j in range(n)]
                b[i] -= f * b[col]
    ak = [b[i] / A[i][i] for i in range(n)]
    a0 = -2 * sum(ak)
    return [a0] + ak


def coefficients(r: int) -> np.ndarray:
    return np.array([float(f) for f in stencil_coefficients(r)], dtype=np.float64)


def symbol(theta, r: int):
    """1D Fourier symbol of the stencil: ``a0 + 2 sum_k a_k cos(k theta)``
    (the eigenvalue of the 1D stencil on ``exp(i k x)``, times h^2)."""
    a = coefficients(r)
    theta = np.asarray(theta, dtype=np.float64)
    s = np.full_like(theta, a[0])
    for k in range(1, r + 1):
        s = s + 2.0 * a[k] * np.cos(k * theta)
    return s


def stability_limit(r: int) -> float:
    """Largest ``v dt / dx`` for which the 3D leapfrog is stable.

    A Fourier mode grows iff ``(v dt/dx)^2 * (-sum_axes symbol) > 4``; the
    largest ``-symbol`` over theta in [0, pi] is found on a fine grid (for
    these weights it is at theta = pi).
    """
    theta = np.linspace(0.0, math.pi, 20001)
    smax = float(np.max(-symbol(theta, r)))
    return 2.0 / math.sqrt(3.0 * smax)


# ----------------------------------------------------------------------------
# model preparation, sponge, wavelet, geometry
# ----------------------------------------------------------------------------

SPONGE_ALPHA = 0.015  # Cerjan et al. (1985) damping per cell


def sponge_profile(n_padded: int, nb: int) -> np.ndarray:
    """1D sponge factor along one axis of length ``n_padded``.

    A cell at distance ``d`` cells from the nearer outer face (d = 0 on the
    face) with ``d < nb`` gets ``exp(-(alpha (nb - d))^2)``; all other cells
    get exactly 1. The 3D factor is the product of the three axis profiles.
    """
    g = np.ones(n_padded, dtype=np.float64)
    for i in range(n_padded):
        d = min(i, n_padded - 1 - i)
        if d < nb:
            g[i] = math.exp(-(SPONGE_ALPHA * (nb - d)) ** 2)
    return g


def pad_model(m: np.ndarray, nb: int) -> np.ndarray:
    """Extend a model-grid array by ``nb`` cells on all six faces, each
    padded cell taking the value of the nearest model cell."""
    return np.pad(np.asarray(m, dtype=np.float64), nb, mode="edge")


def model_c(vel: np.ndarray, nb: int, dt: float, squared: bool = False) -> np.ndarray:
    """``c = v^2 dt^2`` on the padded grid from a model-grid velocity
    (``squared=True``: the input already is v^2)."""
    v2 = np.asarray(vel, dtype=np.float64)
    if not squared:
        v2 = v2 * v2
    return pad_model(v2, nb) * (dt * dt)


def fold_padding(gp: np.ndarray, nb: int) -> np.ndarray:
    """Transpose of ``pad_model``: every padded cell adds its value to the
    model cell it was copied from."""
    NZ, NY, NX = gp.shape
    nz, ny, nx = NZ - 2 * nb, NY - 2 * nb, NX - 2 * nb
    out = np.zeros((nz, ny, nx), dtype=np.float64)
    src_z = np.clip(np.arange(NZ) - nb, 0, nz - 1)
    src_y = np.clip(np.arange(NY) - nb, 0, ny - 1)
    src_x = np.clip(np.arange(NX) - nb, 0, nx - 1)
    for z in range(NZ):
        for y in range(NY):
            np.add.at(out[src_z[z], src_y[y]], src_x, gp[z, y])
    return out


def ricker(nt: int, dt: float, f0: float, t0: float) -> np.ndarray:
    """Ricker wavelet samples ``w^n = w(n dt)``, n = 0..nt-1."""
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def padded_index(coords: np.ndarray, nb: int, padded_shape) -> np.ndarray:
    """Linear padded-grid indices of model coordinates ``[n][3]`` (x, y, z)."""
    NZ, NY, NX = padded_shape
    c = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
    return np.ascontiguousarray(((c[:, 2] + nb) * NY + (c[:, 1] + nb)) * NX + (c[:, 0] + nb))


# ----------------------------------------------------------------------------
# the discrete operators
# ----------------------------------------------------------------------------

class Grid:
    """Padded grid with its coefficient ``c = v^2 dt^2`` and sponge."""

    def __init__(self, c: np.ndarray, nb: int, r: int, dx: float,
                 sponge: bool = True, profiles=None):
        """``profiles = (gx, gy, gz)`` overrides the sponge profiles (a crop of
        a larger grid keeps the profiles of the grid it was cut from)."""
        self.c = np.ascontiguousarray(c, dtype=np.float64)
        self.NZ, self.NY, self.NX = self.c.shape
        self.nb, self.r, self.dx = int(nb), int(r), float(dx)
        self.a = np.ascontiguousarray(coefficients(r))
        nbs = self.nb if sponge else 0
        if profiles is None:
            self.gx = sponge_profile(self.NX, nbs)
            self.gy = sponge_profile(self.NY, nbs)
            self.gz = sponge_profile(self.NZ, nbs)
        else:
            self.gx, self.gy, self.gz = (np.ascontiguousarray(g, dtype=np.float64)
                                         for g in profiles)
            assert (self.gx.size, self.gy.size, self.gz.size) == (self.NX, self.NY, self.NZ)
        self._s = _Grid(self.NX, self.NY, self.NZ, self.nb, self.r, self.dx,
                        _ptr(self.a), _ptr(self.c), _ptr(self.gx), _ptr(self.gy),
                        _ptr(self.gz))

    @property
    def shape(self):
        return (self.NZ, self.NY, self.NX)

    @property
    def model_shape(self):
        return (self.NZ - 2 * self.nb, self.NY - 2 * self.nb, self.NX - 2 * self.nb)

    def g(self) -> np.ndarray:
        return self.gz[:, None, None] * self.gy[None, :, None] * self.gx[None, None, :]

    def laplacian(self, u: np.ndarray) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.shape == self.shape
        out = np.empty_like(u)
        _load().orc_laplacian(ctypes.byref(self._s), _ptr(u), _ptr(out))
        return out

    def step(self, u_cur: np.ndarray, u_prev: np.ndarray) -> np.ndarray:
        """One source-free leapfrog step: ``g (2u + c L u) - g^2 u_prev``."""
        u_cur = np.ascontiguousarray(u_cur, dtype=np.float64)
        u_prev = np.ascontiguousarray(u_prev, dtype=np.float64)
        out = np.empty_like(u_cur)
        _load().orc_step(ctypes.byref(self._s), _ptr(u_cur), _ptr(u_prev), _ptr(out))
        return out

    def forward(self, w: np.ndarray, src: int, rec: np.ndarray, keep_u: bool = False,
                keep_lu: bool = False, keep_last: bool = False) -> Dict[str, np.ndarray]:
        """Forward modelling (see ``orc_forward``); ``src``/``rec`` are linear
        padded indices. Returns ``data [nt][nrec]`` and, on request, the model
        region snapshots ``u [nt]`` (u^{n+1}), ``lu [nt]`` (L u^n) and the last
        two fields ``last = (u^{nt-1}, u^{nt})``."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        rec = np.ascontiguousarray(rec, dtype=np.int64)
        nt, nrec = w.shape[0], rec.shape[0]
        data = np.zeros((nt, nrec))
        out = {"data": data}
        if keep_u:
            out["u"] = np.zeros((nt,) + self.model_shape)
        if keep_lu:
            out["lu"] = np.zeros((nt,) + self.shape)
        if keep_last:
            out["last"] = np.zeros((2,) + self.shape)
        rc = _load().orc_forward(ctypes.byref(self._s), nt, _ptr(w), int(src), nrec,
                                 _ptr(rec), _ptr(data), _ptr(out.get("u")),
                                 _ptr(out.get("lu")), _ptr(out.get("last")))
        if rc != 0:
            raise MemoryError("oracle forward: allocation failed")
        return out

    def adjoint(self, w: np.ndarray, src: int, rec: np.ndarray, resid: np.ndarray,
                snap_u: Optional[np.ndarray] = None, image_every: int = 1,
                snap_lu: Optional[np.ndarray] = None, keep_last: bool = False
                ) -> Dict[str, np.ndarray]:
        """Receiver propagation backward in time (see ``orc_adjoint``).
        Returns ``src_adj [nt]`` and, when the snapshots are given, ``image``
        (model region) and ``grad_acc`` (padded)."""
        if image_every < 1:
            raise ValueError("image_every must be >= 1")
        w = np.ascontiguousarray(w, dtype=np.float64)
        rec = np.ascontiguousarray(rec, dtype=np.int64)
        resid = np.ascontiguousarray(resid, dtype=np.float64)
        nt, nrec = w.shape[0], rec.shape[0]
        assert resid.shape == (nt, nrec)
        out = {"src_adj": np.zeros(nt)}
        if snap_u is not None:
            snap_u = np.ascontiguousarray(snap_u, dtype=np.float64)
            out["image"] = np.zeros(self.model_shape)
        if snap_lu is not None:
            snap_lu = np.ascontiguousarray(snap_lu, dtype=np.float64)
            out["grad_acc"] = np.zeros(self.shape)
        if keep_last:
            out["last"] = np.zeros((2,) + self.shape)
        rc = _load().orc_adjoint(ctypes.byref(self._s), nt, _ptr(w), int(src), nrec,
                                 _ptr(rec), _ptr(resid), _ptr(snap_u), int(image_every),
                                 _ptr(out.get("image")), _ptr(snap_lu),
                                 _ptr(out.get("grad_acc")), _ptr(out["src_adj"]),
                                 _ptr(out.get("last")))
        if rc != 0:
            raise MemoryError("oracle adjoint: allocation failed")
        return out


# ----------------------------------------------------------------------------
# whole problems
# ----------------------------------------------------------------------------

class Problem:
    """One shot: model, discretisation and geometry, all in FP64."""

    def __init__(self, vel: np.ndarray, nb: int, r: int, dx: float, dt: float,
                 nt: int, f0: float, t0: float, src_xyz, rec_xyz: np.ndarray,
                 squared: bool = False, sponge: bool = True):
        self.nb, self.r, self.dx, self.dt, self.nt = nb, r, dx, dt, nt
        self.f0, self.t0 = f0, t0
        self.squared = squared
        self.vel = np.asarray(vel, dtype=np.float64)
        self.grid = Grid(model_c(self.vel, nb, dt, squared), nb, r, dx, sponge)
        self.w = ricker(nt, dt, f0, t0)
        self.src = int(padded_index(np.array(src_xyz).reshape(1, 3), nb, self.grid.shape)[0])
        self.rec = padded_index(rec_xyz, nb, self.grid.shape)

    def forward(self, **kw):
        return self.grid.forward(self.w, self.src, self.rec, **kw)

    def rtm_image(self, d_obs: np.ndarray, image_every: int = 1) -> Dict[str, np.ndarray]:
        """Zero-lag RTM image of ``d_obs``: forward source propagation, then
        receiver propagation of ``d_obs`` with the imaging condition."""
        fw = self.forward(keep_u=True)
        bw = self.grid.adjoint(self.w, self.src, self.rec, d_obs, snap_u=fw["u"],
                               image_every=image_every)
        return {"data": fw["data"], "image": bw["image"], "src_adj": bw["src_adj"]}

    def misfit(self, d_obs: np.ndarray) -> float:
        d = self.forward()["data"]
        return 0.5 * float(np.sum((d - d_obs) ** 2))

    def misfit_and_grad(self, d_obs: np.ndarray):
        """``J = 1/2 ||d - d_obs||^2`` and ``dJ/d(v^2)`` on the model grid
        (``dJ/dv`` chained through v^2 when the velocity is given as v)."""
        fw = self.forward(keep_lu=True)
        resid = fw["data"] - d_obs
        J = 0.5 * float(np.sum(resid * resid))
        bw = self.grid.adjoint(self.w, self.src, self.rec, resid, snap_lu=fw["lu"])
        dx3 = self.dx ** 3
        grad_c = dx3 * bw["grad_acc"] / self.grid.c
        grad_v2 = fold_padding(grad_c, self.nb) * (self.dt * self.dt)
        return J, grad_v2
