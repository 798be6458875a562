"""FP64 oracle of the snapshot-compression autoencoder -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and the CPU legs of ``bench.py`` use it; the CUDA path never
does. The paper has no learned component; the network follows the learned
snapshot-compression reading of the workload: a 4-layer 3D convolutional
autoencoder that compresses a source-wavefield snapshot 8x (float32 voxels to
a bfloat16 latent of 16 channels on a 4x coarser grid) for the imaging
condition. Layers (activations channels-last, [z][y][x][c]):

* normalise: ``x0 = s / rms(s)``
* E1 patch conv 1 -> 32, kernel 2, stride 2, + LeakyReLU(0.1)
* E2 conv 32 -> 16, kernel 3, stride 2, padding 1           (the latent)
* D1 transposed conv 16 -> 32, kernel 4, stride 2, padding 1, + LeakyReLU(0.1)
* D2 transposed patch conv 32 -> 1, kernel 2, stride 2
* de-normalise: ``s_hat = rms(s) * y``

Every product is formed in FP64 from operands rounded to bfloat16 (round to
nearest even) exactly where the GPU stores bfloat16: the normalised input,
the weights, the E1 output, the latent and the D1 output. ``bf16=False``
turns the rounding off (for finite-difference checks of the hand-written
backward pass). Parameters are dicts of FP64 arrays:

* ``W1 [32][2][2][2]``, ``b1 [32]``
* ``W2 [16][3][3][3][32]``, ``b2 [16]``     (out, kz, ky, kx, in)
* ``W3 [32][4][4][4][16]``, ``b3 [32]``     (out, kz, ky, kx, in) of the transposed conv
* ``W4 [2][2][2][32]``, ``b4 [1]``          (dz, dy, dx, in)
"""
from __future__ import annotations

import math
from typing import Dict, Tuple

import numpy as np

C1, C2 = 32, 16
SLOPE = 0.1


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def _q(a, bf16):
    return bf16_round(a) if bf16 else np.asarray(a, dtype=np.float64)


def leaky(a):
    return np.where(a > 0, a, SLOPE * a)


def leaky_grad(a):
    return np.where(a > 0, 1.0, SLOPE)


def init_params(seed: int = 0) -> Dict[str, np.ndarray]:
    """Seeded initial parameters: the random draws come from the shared input
    module (they are inputs of training, not arithmetic of the network)."""
    import rtm_inputs

    return rtm_inputs.ae_init_params(seed)


# ----------------------------------------------------------------------------
# layers (forward and hand-written backward)
# ----------------------------------------------------------------------------

def e1_forward(x0, W1, b1):
    """Patch conv: a[z,y,x,c] = b1[c] + sum_{d in {0,1}^3} W1[c,d] x0[2z+dz, 2y+dy, 2x+dx]."""
    Z, Y, X = x0.shape
    a = np.broadcast_to(b1, (Z // 2, Y // 2, X // 2, C1)).copy()
    for dz in range(2):
        for dy in range(2):
            for dx in range(2):
                a += x0[dz::2, dy::2, dx::2][..., None] * W1[:, dz, dy, dx]
    return a


def e1_backward(x0, W1, ga):
    """Gradients of e1_forward w.r.t. x0, W1, b1 given dL/da."""
    gx = np.zeros(x0.shape)
    gW = np.zeros_like(W1)
    for dz in range(2):
        for dy in range(2):
            for dx in range(2):
                xs = x0[dz::2, dy::2, dx::2]
                gW[:, dz, dy, dx] = np.einsum("zyxc,zyx->c", ga, xs)
                gx[dz::2, dy::2, dx::2] = ga @ W1[:, dz, dy, dx]
    return gx, gW, ga.sum(axis=(0, 1, 2))


def _pad1(h):
    return np.pad(h, ((1, 1), (1, 1), (1, 1), (0, 0)))


def e2_forward(h1, W2, b2):
    """Strided conv: lat[z,y,x,o] = b2[o] + sum_{k in {0,1,2}^3} sum_i
    W2[o,k,i] h1[2z+kz-1, 2y+ky-1, 2x+kx-1, i] (zero outside)."""
    mz, my, mx = (d // 2 for d in h1.shape[:3])
    hp = _pad1(h1)
    lat = np.broadcast_to(b2, (mz, my, mx, C2)).copy()
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                win = hp[kz:kz + 2 * mz:2, ky:ky + 2 * my:2, kx:kx + 2 * mx:2]
                lat += win @ W2[:, kz, ky, kx].T
    return lat


def e2_backward(h1, W2, glat):
    mz, my, mx = (d // 2 for d in h1.shape[:3])
    hp = _pad1(h1)
    ghp = np.zeros_like(hp)
    gW = np.zeros_like(W2)
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                sl = (slice(kz, kz + 2 * mz, 2), slice(ky, ky + 2 * my, 2),
                      slice(kx, kx + 2 * mx, 2))
                gW[:, kz, ky, kx] = np.einsum("zyxo,zyxi->oi", glat, hp[sl])
                ghp[sl] += glat @ W2[:, kz, ky, kx]
    return ghp[1:-1, 1:-1, 1:-1], gW, glat.sum(axis=(0, 1, 2))


def _convt_taps(q: int):
    """Transposed conv, kernel 4, stride 2, padding 1: output 2j+q receives
    input j + t with kernel index k, for the two (t, k) pairs of parity q."""
    return [(0, 1), (-1, 3)] if q == 0 else [(1, 0), (0, 2)]


def d1_forward(lat, W3, b3):
    """Transposed conv: g[o] = b3 + sum over (i, k) with o = 2i + k - 1 of
    W3[.,k,.] lat[i] (zero outside), per axis."""
    mz, my, mx = lat.shape[:3]
    lp = np.pad(lat, ((1, 1), (1, 1), (1, 1), (0, 0)))
    g = np.broadcast_to(b3, (2 * mz, 2 * my, 2 * mx, C1)).copy()
    for qz in range(2):
        for qy in range(2):
            for qx in range(2):
                acc = np.zeros((mz, my, mx, C1))
                for tz, kz in _convt_taps(qz):
                    for ty, ky in _convt_taps(qy):
                        for tx, kx in _convt_taps(qx):
                            win = lp[1 + tz:1 + tz + mz, 1 + ty:1 + ty + my, 1 + tx:1 + tx + mx]
                            acc += win @ W3[:, kz, ky, kx].T
                g[qz::2, qy::2, qx::2] += acc
    return g


def d1_backward(lat, W3, gg):
    mz, my, mx = lat.shape[:3]
    lp = np.pad(lat, ((1, 1), (1, 1), (1, 1), (0, 0)))
    glp = np.zeros_like(lp)
    gW = np.zeros_like(W3)
    for qz in range(2):
        for qy in range(2):
            for qx in range(2):
                go = gg[qz::2, qy::2, qx::2]
                for tz, kz in _convt_taps(qz):
                    for ty, ky in _convt_taps(qy):
                        for tx, kx in _convt_taps(qx):
                            sl = (slice(1 + tz, 1 + tz + mz), slice(1 + ty, 1 + ty + my),
                                  slice(1 + tx, 1 + tx + mx))
                            win = lp[sl]
                            gW[:, kz, ky, kx] += np.einsum("zyxo,zyxi->oi", go, win)
                            glp[sl] += go @ W3[:, kz, ky, kx]
    return glp[1:-1, 1:-1, 1:-1], gW, gg.sum(axis=(0, 1, 2))


def d2_forward(g1, W4, b4):
    """Transposed patch conv: y[2z+dz, 2y+dy, 2x+dx] = b4 + sum_i W4[d,i] g1[z,y,x,i]."""
    mz, my, mx = g1.shape[:3]
    y = np.empty((2 * mz, 2 * my, 2 * mx))
    for dz in range(2):
        for dy in range(2):
            for dx in range(2):
                y[dz::2, dy::2, dx::2] = g1 @ W4[dz, dy, dx] + b4[0]
    return y


def d2_backward(g1, W4, gy):
    gg = np.zeros_like(g1)
    gW = np.zeros_like(W4)
    for dz in range(2):
        for dy in range(2):
            for dx in range(2):
                go = gy[dz::2, dy::2, dx::2]
                gW[dz, dy, dx] = np.einsum("zyx,zyxi->i", go, g1)
                gg += go[..., None] * W4[dz, dy, dx]
    return gg, gW, np.array([gy.sum()])


# ----------------------------------------------------------------------------
# the network
# ----------------------------------------------------------------------------

def rms(s) -> float:
    return float(np.sqrt(np.mean(np.asarray(s, np.float64) ** 2)))


def forward(params, x0, bf16: bool = True, keep: bool = False):
    """Normalised input x0 [N][N][N] -> reconstruction y (normalised)."""
    q = lambda a: _q(a, bf16)  # noqa: E731
    P = {k: (q(v) if k.startswith("W") else np.asarray(v, np.float64)) for k, v in params.items()}
    xq = q(x0)
    a1 = e1_forward(xq, P["W1"], P["b1"])
    h1 = q(leaky(a1))
    lat = q(e2_forward(h1, P["W2"], P["b2"]))
    a3 = d1_forward(lat, P["W3"], P["b3"])
    g1 = q(leaky(a3))
    y = d2_forward(g1, P["W4"], P["b4"])
    if keep:
        return y, dict(P=P, xq=xq, a1=a1, h1=h1, lat=lat, a3=a3, g1=g1)
    return y


def encode(params, s, bf16=True):
    """Snapshot -> (latent, scale)."""
    sc = rms(s)
    x0 = np.asarray(s, np.float64) / (sc if sc > 0 else 1.0)
    q = lambda a: _q(a, bf16)  # noqa: E731
    P = {k: (q(v) if k.startswith("W") else np.asarray(v, np.float64)) for k, v in params.items()}
    h1 = q(leaky(e1_forward(q(x0), P["W1"], P["b1"])))
    return q(e2_forward(h1, P["W2"], P["b2"])), sc


def decode(params, lat, sc, bf16=True):
    q = lambda a: _q(a, bf16)  # noqa: E731
    P = {k: (q(v) if k.startswith("W") else np.asarray(v, np.float64)) for k, v in params.items()}
    g1 = q(leaky(d1_forward(lat, P["W3"], P["b3"])))
    return sc * d2_forward(g1, P["W4"], P["b4"])


def loss_and_grads(params, x0, bf16: bool = True, bf16_grads: bool = False,
                   scale: float = 1.0) -> Tuple[float, Dict[str, np.ndarray]]:
    """MSE ``mean((y - x0)^2)`` and its gradients with respect to every
    parameter (straight through the bfloat16 roundings).

    ``bf16_grads`` also rounds the back-propagated gradients to bfloat16 at
    the four points where the GPU feeds them to the tensor cores: dL/dy,
    dL/d(a3), dL/d(latent) and dL/d(a1); bias gradients are then sums of
    those rounded tensors. ``scale`` multiplies dL/dy (a batch of B samples
    averages with scale = 1/B)."""
    y, t = forward(params, x0, bf16, keep=True)
    P = t["P"]
    n = y.size
    diff = y - x0
    L = float(np.mean(diff * diff))
    qg = (lambda a: bf16_round(a)) if bf16_grads else (lambda a: a)  # noqa: E731
    gy = qg(scale * 2.0 * diff / n)
    gg1, gW4, gb4 = d2_backward(t["g1"], P["W4"], gy)
    ga3 = qg(gg1 * leaky_grad(t["a3"]))
    glat, gW3, gb3 = d1_backward(t["lat"], P["W3"], ga3)
    glat = qg(glat)
    gh1, gW2, gb2 = e2_backward(t["h1"], P["W2"], glat)
    ga1 = qg(gh1 * leaky_grad(t["a1"]))
    _, gW1, gb1 = e1_backward(t["xq"], P["W1"], ga1)
    return L, {"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3,
               "W4": gW4, "b4": gb4}


PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


def flatten(params) -> np.ndarray:
    """Parameters as one flat vector in the fixed order W1 b1 W2 b2 W3 b3 W4 b4
    (each array in C order)."""
    return np.concatenate([np.asarray(params[k], np.float64).ravel() for k in PARAM_ORDER])


def unflatten(vec) -> Dict[str, np.ndarray]:
    shapes = {k: v.shape for k, v in init_params(0).items()}
    out, o = {}, 0
    for k in PARAM_ORDER:
        sz = int(np.prod(shapes[k]))
        out[k] = np.asarray(vec[o:o + sz], np.float64).reshape(shapes[k])
        o += sz
    return out


def adam_step(params, grads, state, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
              clip=None):
    """One Adam update (Kingma and Ba, 2015) at step t >= 1, in place. With
    ``clip`` the gradients are first scaled so that their joint L2 norm over
    all parameters is at most ``clip``."""
    scale = 1.0
    if clip:
        norm = math.sqrt(sum(float(np.sum(np.asarray(g, np.float64) ** 2)) for g in grads.values()))
        if norm > clip:
            scale = clip / norm
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        g = grads[k] * scale
        m[...] = beta1 * m + (1 - beta1) * g
        v[...] = beta2 * v + (1 - beta2) * g * g
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params


def decimate(s):
    """Non-learned 8x baseline: keep every other sample on each axis (FP32)."""
    return np.asarray(s, np.float64)[::2, ::2, ::2].astype(np.float32).astype(np.float64)


def trilinear_upsample(d, N):
    """Linear interpolation of a decimated field back to N samples per axis
    (sample 2i holds d[i]; the last odd sample copies its left neighbour).
    N is one size for all three axes or a (nz, ny, nx) triple."""
    out = np.asarray(d, np.float64)
    sizes = (N, N, N) if np.isscalar(N) else tuple(N)
    for axis in range(3):
        N = sizes[axis]
        n = out.shape[axis]
        shape = list(out.shape)
        shape[axis] = N
        up = np.zeros(shape)
        ev = [slice(None)] * 3
        od = [slice(None)] * 3
        ev[axis] = slice(0, 2 * n, 2)
        up[tuple(ev)] = out
        left = np.take(out, np.arange(0, n - 1), axis=axis)
        right = np.take(out, np.arange(1, n), axis=axis)
        od[axis] = slice(1, 2 * n - 1, 2)
        up[tuple(od)] = 0.5 * (left + right)
        if N == 2 * n:
            last = [slice(None)] * 3
            last[axis] = slice(N - 1, N)
            up[tuple(last)] = np.take(out, [n - 1], axis=axis)
        out = up
    return out
