"""GPU parity of the tensor-core snapshot codec against the FP64 autoencoder
oracle, which rounds to bfloat16 exactly where the GPU stores bfloat16.

Tolerance: a bfloat16 value is exact to 2^-9 relative; the GPU accumulates
in float32 and the oracle in float64, so a stored bfloat16 intermediate can
land one bfloat16 step away where the two sums straddle a rounding boundary
(rare). Such flips leave relative L2 errors far below 2e-3, the bar used for
every codec quantity below."""
import numpy as np
import pytest

import rtm_inputs
from helpers import rel_l2

pytestmark = pytest.mark.gpu
TOL = 2e-3


def _snapshot(shape=(32, 32, 32), nt=70, seed=1):
    """A wavefield snapshot from the oracle's propagator (model region)."""
    import oracle

    nz, ny, nx = shape
    v = rtm_inputs.smooth_random_velocity(nx, ny, nz, 3.0, 1500.0, 3000.0, seed=seed)
    rec = rtm_inputs.surface_receivers(nx, ny, 2, stride=8)
    p = oracle.Problem(v, 6, 4, 10.0, rtm_inputs.courant_dt(10.0, 3000.0), nt, 30.0, 0.035,
                       (nx // 2, ny // 2, nz // 3), rec)
    return p.forward(keep_u=True)["u"][-1]


def _params(seed=3):
    return rtm_inputs.ae_flat(rtm_inputs.ae_init_params(seed))


def _cuda(a, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to(device="cuda", dtype=dtype or torch.float32)


@pytest.mark.parametrize("N", [16, 32])
@pytest.mark.parametrize("M,K", [(128, 32), (300, 96), (1000, 864)])
def test_tensor_core_gemm_matches_numpy(M, K, N):
    import torch

    from oracle import ae as oae
    from paper_1603_03971_gb300 import codec

    rng = np.random.default_rng(M + K + N)
    A = oae.bf16_round(rng.standard_normal((M, K)))
    B = oae.bf16_round(rng.standard_normal((N, K)))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = codec.gemm_bf16(_cuda(A, torch.bfloat16), _cuda(B, torch.bfloat16), status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = A @ B.T
    np.testing.assert_allclose(C.cpu().numpy(), ref, rtol=1e-5, atol=1e-4 * np.abs(ref).max())


def test_encode_decode_match_oracle():
    import torch

    from oracle import ae as oae
    from paper_1603_03971_gb300 import codec

    s = _snapshot()
    P = _params()
    ws = codec.alloc_workspace(s.shape)
    lat, sc = codec.encode(_cuda(P), _cuda(s), ws)
    torch.cuda.synchronize()
    lat_ref, sc_ref = oae.encode(oae.unflatten(P), s.astype(np.float32).astype(np.float64))
    assert float(sc.item()) == pytest.approx(sc_ref, rel=1e-6)
    assert rel_l2(lat.float().cpu().numpy(), lat_ref) <= TOL
    # decode the GPU latent on both sides
    out = codec.decode(_cuda(P), lat, sc, ws)
    torch.cuda.synchronize()
    ref = oae.decode(oae.unflatten(P), lat.float().cpu().numpy().astype(np.float64),
                     float(sc.item()))
    assert rel_l2(out.cpu().numpy(), ref) <= TOL


def test_strided_snapshot_views_encode_identically():
    """The codec reads and writes strided views (the model region inside a
    padded slab) exactly as dense arrays."""
    import torch

    from paper_1603_03971_gb300 import codec

    s = _snapshot((16, 24, 20), nt=50, seed=2)
    P = _cuda(_params(4))
    ws = codec.alloc_workspace(s.shape)
    dense = _cuda(s)
    big = torch.full((16, 24, 20 + 12), float("nan"), device="cuda")
    big[:, :, 5:25] = dense
    view = big[:, :, 5:25]
    l1, s1 = codec.encode(P, dense, ws)
    l2, s2 = codec.encode(P, view, ws)
    torch.cuda.synchronize()
    assert torch.equal(l1, l2) and torch.equal(s1, s2)
    o1 = codec.decode(P, l1, s1, ws)
    out = torch.full_like(big, 7.0)
    codec.decode(P, l1, s1, ws, out=out[:, :, 5:25])
    torch.cuda.synchronize()
    assert torch.equal(out[:, :, 5:25], o1)
    assert bool((out[:, :, :5] == 7.0).all()) and bool((out[:, :, 25:] == 7.0).all())


@pytest.mark.parametrize("shape", [(4, 4, 4), (32, 32, 32), (20, 28, 36), (160, 96, 72)])
def test_marching_decoder_equals_gemm_decoder(shape):
    """The z-marching decoder (TMA plane loads read in place by the tensor
    cores, several z chunks and ragged x / y columns at the largest shape)
    and the GEMM-engine decoder: the same bfloat16 g1 and weights, D1 summed
    in the same order; D2's 32 products are exact in float32 and summed by
    the tensor cores in the marching decoder, sequentially in the other, so
    the outputs agree to float32 rounding of a 32-term sum. The strided
    output (rows not 16-byte aligned) equals the dense one exactly and leaves
    the columns beside it untouched."""
    import torch

    from paper_1603_03971_gb300 import codec

    nz, ny, nx = shape
    P = _cuda(_params(5))
    lat = _cuda(0.5 * rtm_inputs.standard_normal((nz // 4, ny // 4, nx // 4, 16), 61),
                torch.bfloat16)
    sc = torch.tensor([1.7], device="cuda")
    ws = codec.alloc_workspace(shape)
    try:
        codec.set_decoder("gemm")
        ref = codec.decode(P, lat, sc, ws)
        codec.set_decoder("march")
        out = codec.decode(P, lat, sc, ws)
        big = torch.full((nz, ny, nx + 5), float("nan"), device="cuda")
        codec.decode(P, lat, sc, ws, out=big[:, :, 1:1 + nx])
        torch.cuda.synchronize()
    finally:
        codec.set_decoder("auto")
    import paper_1603_03971_gb300 as rtm

    rtm.check(ws)
    scale = float(ref.abs().max())
    assert scale > 0
    assert float((out - ref).abs().max()) <= 2e-6 * scale
    assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-6
    assert torch.equal(big[:, :, 1:1 + nx], out)
    assert bool(big[:, :, 0].isnan().all()) and bool(big[:, :, 1 + nx:].isnan().all())


@pytest.mark.parametrize("shape", [(4, 4, 4), (32, 32, 32), (20, 28, 36), (160, 96, 72)])
def test_marching_encoder_equals_gemm_encoder(shape):
    """The z-marching encoder (h1 kept in shared memory, E1 and E2 on the
    tensor cores reading operands in place) forms the same products and sums
    in the same order as the GEMM-engine encoder: equal latents and scales,
    and both match the oracle."""
    import torch

    from oracle import ae as oae
    from paper_1603_03971_gb300 import codec

    nz, ny, nx = shape
    P = _params(6)
    s = rtm_inputs.standard_normal(shape, 62, np.float32)
    s[nz // 2:] *= 3.0  # a scale jump, so that rms normalisation matters
    Pd, sd = _cuda(P), _cuda(s)
    ws = codec.alloc_workspace(shape)
    try:
        codec.set_encoder("gemm")
        l_ref, sc_ref = codec.encode(Pd, sd, ws)
        codec.set_encoder("march")
        l_new, sc_new = codec.encode(Pd, sd, ws)
        torch.cuda.synchronize()
    finally:
        codec.set_encoder("auto")
    import paper_1603_03971_gb300 as rtm

    rtm.check(ws)
    assert torch.equal(sc_new, sc_ref)
    assert torch.equal(l_new, l_ref)
    lat_or, _ = oae.encode(oae.unflatten(P), s.astype(np.float64))
    assert rel_l2(l_new.float().cpu().numpy(), lat_or) <= TOL


@pytest.mark.parametrize("shape", [(16, 16, 16), (20, 12, 24)])
def test_training_gradient_matches_oracle(shape):
    import torch

    from oracle import ae as oae
    from paper_1603_03971_gb300 import codec

    batch = np.stack([_snapshot(shape, nt=45 + 10 * i, seed=5 + i) for i in range(2)])
    P = _params(6)
    ws = codec.alloc_workspace(shape)
    grad = torch.zeros(codec.NPARAMS, device="cuda")
    loss = codec.train_step(_cuda(P), None, None, 0, 0.0, _cuda(batch), ws, grad_out=grad)
    torch.cuda.synchronize()
    params = oae.unflatten(P)
    L_ref, g_ref = 0.0, None
    for b in batch:
        s = b.astype(np.float32).astype(np.float64)
        x0 = s / oae.rms(s)
        L, g = oae.loss_and_grads(params, x0, bf16=True, bf16_grads=True, scale=0.5)
        L_ref += 0.5 * L
        g_ref = g if g_ref is None else {k: g_ref[k] + g[k] for k in g}
    assert float(loss.item()) == pytest.approx(L_ref, rel=1e-4)
    gg = oae.unflatten(grad.cpu().numpy().astype(np.float64))
    for k in oae.PARAM_ORDER:
        assert rel_l2(gg[k], g_ref[k]) <= 5e-3, k


def test_adam_step_matches_oracle():
    import torch

    from oracle import ae as oae
    from paper_1603_03971_gb300 import codec

    shape = (16, 16, 16)
    batch = _snapshot(shape, nt=55, seed=9)[None]
    P0 = _params(7)
    P = _cuda(P0)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    ws = codec.alloc_workspace(shape)
    grad = torch.zeros_like(P)
    codec.train_step(P, m, v, 1, 1e-3, _cuda(batch), ws, grad_out=grad)
    torch.cuda.synchronize()
    g = grad.cpu().numpy().astype(np.float64)
    ref = {"w": P0.astype(np.float32).astype(np.float64)}
    oae.adam_step(ref, {"w": g}, {}, 1, lr=1e-3, clip=1.0)
    np.testing.assert_allclose(P.cpu().numpy(), ref["w"], rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("shape", [(160, 96, 72), (48, 72, 136)])
def test_marching_codec_matches_oracle_at_full_scheduling_size(shape):
    """The z-marching encoder and decoder that the learned RTM shot runs,
    each against the FP64 oracle, element by element, at sizes that reach
    their full scheduling paths: several latent columns in x and y with
    ragged last columns (72 -> 18 and 136 -> 34 latent x points against
    16-point columns; 96 -> 24 and 72 -> 18 latent y points against 8-row
    columns) and several z chunks per column."""
    import torch

    from oracle import ae as oae
    from paper_1603_03971_gb300 import codec

    nz, ny, nx = shape
    P = _params(8)
    s = rtm_inputs.standard_normal(shape, 63, np.float32)
    s[:, :, nx // 3:] *= 2.5  # a scale jump across columns
    Pd = _cuda(P)
    ws = codec.alloc_workspace(shape)
    try:
        codec.set_encoder("march")
        codec.set_decoder("march")
        lat, sc = codec.encode(Pd, _cuda(s), ws)
        out = codec.decode(Pd, lat, sc, ws)
        torch.cuda.synchronize()
    finally:
        codec.set_encoder("auto")
        codec.set_decoder("auto")
    import paper_1603_03971_gb300 as rtm

    rtm.check(ws)
    params = oae.unflatten(P)
    lat_or, sc_or = oae.encode(params, s.astype(np.float64))
    assert float(sc.item()) == pytest.approx(sc_or, rel=1e-6)
    assert rel_l2(lat.float().cpu().numpy(), lat_or) <= TOL
    # the decoder on the GPU's latent, on both sides
    ref = oae.decode(params, lat.float().cpu().numpy().astype(np.float64), float(sc.item()))
    assert rel_l2(out.cpu().numpy(), ref) <= TOL
