"""Pins of the autoencoder oracle: each layer against torch's FP64 CPU
convolution routines (an independent library implementation), the
hand-written backward pass against central finite differences, bfloat16
rounding against torch's conversion, Adam against its closed-form first step
and torch.optim.Adam, and the decimation baseline against exactness on affine
fields."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import ae


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-30, 30, 10000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 65504.0, 1e-40]])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(ae.bf16_round(a), ref)
    assert ae.bf16_round(np.array([1.0 + 2 ** -8]))[0] == 1.0  # tie to even


def test_e1_is_a_stride2_kernel2_conv():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((8, 8, 8))
    W = rng.standard_normal((32, 2, 2, 2))
    b = rng.standard_normal(32)
    ref = F.conv3d(_t(x)[None, None], _t(W)[:, None], _t(b), stride=2)[0]
    np.testing.assert_allclose(ae.e1_forward(x, W, b), ref.permute(1, 2, 3, 0).numpy(),
                               rtol=1e-12, atol=1e-12)


def test_e2_is_a_stride2_padded_conv():
    rng = np.random.default_rng(2)
    h = rng.standard_normal((6, 6, 6, 32))
    W = rng.standard_normal((16, 3, 3, 3, 32))
    b = rng.standard_normal(16)
    ref = F.conv3d(_t(h).permute(3, 0, 1, 2)[None], _t(W).permute(0, 4, 1, 2, 3), _t(b),
                   stride=2, padding=1)[0]
    np.testing.assert_allclose(ae.e2_forward(h, W, b), ref.permute(1, 2, 3, 0).numpy(),
                               rtol=1e-12, atol=1e-11)


def test_d1_is_a_stride2_transposed_conv():
    rng = np.random.default_rng(3)
    lat = rng.standard_normal((3, 3, 3, 16))
    W = rng.standard_normal((32, 4, 4, 4, 16))
    b = rng.standard_normal(32)
    # torch weight layout for conv_transpose3d: [in, out, kz, ky, kx]
    ref = F.conv_transpose3d(_t(lat).permute(3, 0, 1, 2)[None], _t(W).permute(4, 0, 1, 2, 3),
                             _t(b), stride=2, padding=1)[0]
    np.testing.assert_allclose(ae.d1_forward(lat, W, b), ref.permute(1, 2, 3, 0).numpy(),
                               rtol=1e-12, atol=1e-11)


def test_d2_is_a_stride2_kernel2_transposed_conv():
    rng = np.random.default_rng(4)
    g = rng.standard_normal((4, 4, 4, 32))
    W = rng.standard_normal((2, 2, 2, 32))
    b = rng.standard_normal(1)
    ref = F.conv_transpose3d(_t(g).permute(3, 0, 1, 2)[None],
                             _t(W).permute(3, 0, 1, 2)[:, None], _t(b), stride=2)[0, 0]
    np.testing.assert_allclose(ae.d2_forward(g, W, b), ref.numpy(), rtol=1e-12, atol=1e-11)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(5)
    params = ae.init_params(7)
    x0 = rng.standard_normal((8, 8, 8))
    L, grads = ae.loss_and_grads(params, x0, bf16=False)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"):
        d = rng.standard_normal(params[name].shape)
        eps = 1e-6
        pp = {k: v.copy() for k, v in params.items()}
        pm = {k: v.copy() for k, v in params.items()}
        pp[name] = pp[name] + eps * d
        pm[name] = pm[name] - eps * d
        Lp = float(np.mean((ae.forward(pp, x0, bf16=False) - x0) ** 2))
        Lm = float(np.mean((ae.forward(pm, x0, bf16=False) - x0) ** 2))
        fd = (Lp - Lm) / (2 * eps)
        an = float(np.sum(grads[name] * d))
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-12), name


def test_backward_matches_torch_autograd():
    """The same network written with torch's FP64 conv routines and autograd."""
    rng = np.random.default_rng(6)
    params = ae.init_params(8)
    x0 = rng.standard_normal((8, 8, 8))
    L, grads = ae.loss_and_grads(params, x0, bf16=False)
    P = {k: _t(v).requires_grad_(True) for k, v in params.items()}
    x = _t(x0)[None, None]
    h = F.leaky_relu(F.conv3d(x, P["W1"][:, None], P["b1"], stride=2), 0.1)
    lat = F.conv3d(h, P["W2"].permute(0, 4, 1, 2, 3), P["b2"], stride=2, padding=1)
    g = F.leaky_relu(F.conv_transpose3d(lat, P["W3"].permute(4, 0, 1, 2, 3), P["b3"], stride=2,
                                        padding=1), 0.1)
    y = F.conv_transpose3d(g, P["W4"].permute(3, 0, 1, 2)[:, None], P["b4"], stride=2)
    Lt = ((y - x) ** 2).mean()
    Lt.backward()
    assert float(Lt.detach()) == pytest.approx(L, rel=1e-12)
    for k in P:
        np.testing.assert_allclose(grads[k], P[k].grad.numpy(), rtol=1e-9, atol=1e-12)


def test_adam_first_step_closed_form_and_torch():
    rng = np.random.default_rng(9)
    p = {"w": rng.standard_normal(50)}
    g = {"w": rng.standard_normal(50)}
    p0 = p["w"].copy()
    ae.adam_step(p, g, {}, 1, lr=0.01)
    # at t = 1, m_hat = g and v_hat = g^2: the step is lr g / (|g| + eps)
    np.testing.assert_allclose(p["w"], p0 - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8), rtol=1e-12)
    # several steps against torch.optim.Adam
    w = torch.nn.Parameter(_t(p0))
    opt = torch.optim.Adam([w], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    q = {"w": p0.copy()}
    st = {}
    for t in range(1, 6):
        gt = rng.standard_normal(50)
        w.grad = _t(gt)
        opt.step()
        ae.adam_step(q, {"w": gt}, st, t, lr=0.01)
    np.testing.assert_allclose(q["w"], w.detach().numpy(), rtol=1e-10, atol=1e-14)


def test_decimation_baseline_is_exact_on_affine_fields():
    N = 16
    i = np.arange(N, dtype=np.float64)
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    f = 0.5 + 0.25 * x - 0.125 * y + 0.0625 * z
    up = ae.trilinear_upsample(ae.decimate(f), N)
    s = slice(0, N - 1)
    np.testing.assert_allclose(up[s, s, s], f[s, s, s], rtol=0, atol=1e-6)


@pytest.mark.parametrize("shape", [(9, 12, 7), (6, 5, 10), (1, 2, 3)])
def test_decimation_baseline_matches_brute_force_on_non_cubic_grids(shape):
    """The interpolation written as one weighted sum over the eight coarse
    corners of each sample (per axis: an even sample j is the kept sample
    j / 2; an odd one the mean of (j - 1) / 2 and (j + 1) / 2, or a copy of
    (j - 1) / 2 past the last kept sample), sample by sample, against the
    oracle's axis-by-axis sweeps, on odd and even sides."""
    rng = np.random.default_rng(13)
    s = rng.standard_normal(shape)
    d = ae.decimate(s)
    up = ae.trilinear_upsample(d, shape)
    assert d.shape == tuple((n + 1) // 2 for n in shape)

    def taps(j, nc):
        if j % 2 == 0:
            return [(j // 2, 1.0)]
        if (j + 1) // 2 < nc:
            return [((j - 1) // 2, 0.5), ((j + 1) // 2, 0.5)]
        return [((j - 1) // 2, 1.0)]

    ref = np.zeros(shape)
    for z in range(shape[0]):
        for y in range(shape[1]):
            for x in range(shape[2]):
                v = 0.0
                for iz, wz in taps(z, d.shape[0]):
                    for iy, wy in taps(y, d.shape[1]):
                        for ix, wx in taps(x, d.shape[2]):
                            v += wz * wy * wx * d[iz, iy, ix]
                ref[z, y, x] = v
    np.testing.assert_allclose(up, ref, rtol=0, atol=1e-12)
    # the kept samples come back exactly (float32 storage)
    np.testing.assert_array_equal(up[::2, ::2, ::2], s[::2, ::2, ::2].astype(np.float32))


def test_decimation_initialised_network_computes_the_decimation_baseline():
    """The codec's decimation-equivalent initial parameters make the oracle
    network compute decimation + linear interpolation exactly (without
    bfloat16 rounding) away from the upper faces, where the network's
    transposed convolution sees zero padding instead of a copied sample;
    with bfloat16 rounding within 1 %. This also checks the oracle's
    transposed-convolution tap table independently of torch: a wrong (t, k)
    pair breaks the interpolation."""
    from paper_1603_03971_gb300 import learned

    P = ae.unflatten(learned.decimation_init(3).astype(np.float64))
    rng = np.random.default_rng(14)
    for shape in [(16, 16, 16), (12, 8, 20)]:
        s = rng.standard_normal(shape)
        ref = ae.trilinear_upsample(ae.decimate(s), shape)
        inner = tuple(slice(0, n - 1) for n in shape)
        y = ae.forward(P, s, bf16=False)
        np.testing.assert_allclose(y[inner], ref[inner], rtol=0, atol=1e-6)
        yb = ae.forward(P, s, bf16=True)
        err = np.linalg.norm(yb[inner] - ref[inner]) / np.linalg.norm(ref[inner])
        assert err < 1e-2


def test_encode_decode_compress_8x():
    rng = np.random.default_rng(10)
    s = rng.standard_normal((16, 16, 16))
    lat, sc = ae.encode(ae.init_params(1), s)
    assert lat.shape == (4, 4, 4, 16)
    # bfloat16 latent: 2 bytes x 16 channels per 4^3 voxels vs 4 bytes per voxel
    assert (s.size * 4) / (lat.size * 2) == 8.0
    assert ae.decode(ae.init_params(1), lat, sc).shape == s.shape


def test_layers_on_non_cubic_volumes_match_torch():
    rng = np.random.default_rng(11)
    x = rng.standard_normal((12, 8, 16))
    P = ae.init_params(12)
    h = ae.leaky(ae.e1_forward(x, P["W1"], P["b1"]))
    lat = ae.e2_forward(h, P["W2"], P["b2"])
    g = ae.leaky(ae.d1_forward(lat, P["W3"], P["b3"]))
    y = ae.d2_forward(g, P["W4"], P["b4"])
    X = _t(x)[None, None]
    ht = F.leaky_relu(F.conv3d(X, _t(P["W1"])[:, None], _t(P["b1"]), stride=2), 0.1)
    lt = F.conv3d(ht, _t(P["W2"]).permute(0, 4, 1, 2, 3), _t(P["b2"]), stride=2, padding=1)
    gt = F.leaky_relu(F.conv_transpose3d(lt, _t(P["W3"]).permute(4, 0, 1, 2, 3), _t(P["b3"]),
                                         stride=2, padding=1), 0.1)
    yt = F.conv_transpose3d(gt, _t(P["W4"]).permute(3, 0, 1, 2)[:, None], _t(P["b4"]), stride=2)
    np.testing.assert_allclose(y, yt[0, 0].numpy(), rtol=1e-10, atol=1e-10)
    L, grads = ae.loss_and_grads(P, x, bf16=False)
    assert np.isfinite(L) and all(np.isfinite(v).all() for v in grads.values())


def test_adam_with_gradient_clipping_matches_torch():
    rng = np.random.default_rng(13)
    p0 = {"a": rng.standard_normal(20), "b": rng.standard_normal(7)}
    P = {k: torch.nn.Parameter(_t(v)) for k, v in p0.items()}
    opt = torch.optim.Adam(list(P.values()), lr=0.01)
    q = {k: v.copy() for k, v in p0.items()}
    st = {}
    for t in range(1, 6):
        g = {k: rng.standard_normal(v.shape) * 3.0 for k, v in p0.items()}
        for k in P:
            P[k].grad = _t(g[k])
        torch.nn.utils.clip_grad_norm_(list(P.values()), 1.0)
        opt.step()
        ae.adam_step(q, g, st, t, lr=0.01, clip=1.0)
    for k in P:
        np.testing.assert_allclose(q[k], P[k].detach().numpy(), rtol=1e-9, atol=1e-12)
