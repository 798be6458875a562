"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs, element by element (relative L2 <= 1e-4 on wavefields,
data, images and gradients; FP32 fields against FP64)."""
import numpy as np
import pytest

from helpers import Case, DeviceShot, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-4

# shapes chosen to span several tiles (64 x 16 in x-y) with ragged tails and
# to split z into several slabs
SHAPES = {
    "small": dict(nx=28, ny=24, nz=20, nb=6),          # 40 x 36 x 32 padded
    "ragged": dict(nx=100, ny=44, nz=37, nb=10),       # 120 x 64 x 57 padded
    "thin": dict(nx=4, ny=3, nz=5, nb=8, src=(2, 1, 2)),   # 20 x 19 x 21, model smaller than r
}


@pytest.fixture(autouse=True)
def _reset_tuning():
    import paper_1603_03971_gb300 as rtm

    yield
    rtm.set_tuning(4, 0, 0)
    rtm.set_tuning(8, 0, 0)


def test_model_prep_matches_oracle():
    import oracle

    case = Case(**SHAPES["ragged"])
    g = DeviceShot(case)
    c_ref = oracle.model_c(case.velocity(), case.nb, case.dt)
    c = g.c.cpu().numpy()
    assert c.shape == c_ref.shape
    assert np.max(np.abs(c - c_ref) / c_ref) < 3e-7


@pytest.mark.parametrize("r", [4, 8])
@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("zchunk", [0, 16])
def test_forward_parity(r, shape, zchunk):
    import paper_1603_03971_gb300 as rtm

    kw = dict(SHAPES[shape])
    case = Case(r=r, nt=50, **kw)
    if shape == "thin":
        case.rec_stride = 1
    rtm.set_tuning(r, zchunk, 0)
    g = DeviceShot(case)
    data, last = g.forward(keep_last=True)
    ref = case.oracle_problem().forward(keep_last=True)
    assert rel_l2(data.cpu().numpy(), ref["data"]) <= TOL
    assert rel_l2(last[1].cpu().numpy(), ref["last"][1]) <= TOL
    assert rel_l2(last[0].cpu().numpy(), ref["last"][0]) <= TOL


@pytest.mark.parametrize("r", [4, 8])
@pytest.mark.parametrize("storage,ck", [("all", 0), ("ckpt", 16), ("ckpt", 7)])
def test_backward_image_parity(r, storage, ck):
    case = Case(r=r, nt=60, storage=storage, ckpt_every=ck, **SHAPES["ragged"])
    g = DeviceShot(case)
    g.forward()
    d_obs = case.d_obs(g.nrec)
    img, adj = g.backward_image(d_obs, src_adj=True)
    prob = case.oracle_problem()
    fw = prob.forward(keep_u=True)
    bw = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=fw["u"])
    assert rel_l2(img.cpu().numpy(), bw["image"]) <= TOL
    assert rel_l2(adj.cpu().numpy(), bw["src_adj"]) <= TOL


def test_checkpointing_reproduces_store_all_exactly():
    """Segment recompute runs the same kernels on the same values, so the
    checkpointed image equals the store-all image bit for bit."""
    base = dict(r=4, nt=45, **SHAPES["ragged"])
    imgs = []
    for storage, ck in (("all", 0), ("ckpt", 10), ("ckpt", 45), ("ckpt", 1)):
        case = Case(storage=storage, ckpt_every=ck, **base)
        g = DeviceShot(case)
        g.forward()
        img, _ = g.backward_image(case.d_obs(g.nrec))
        imgs.append(img.cpu().numpy())
    for other in imgs[1:]:
        np.testing.assert_array_equal(other, imgs[0])


@pytest.mark.parametrize("storage,ck", [("all", 0), ("ckpt", 12)])
def test_image_every_fourth_step(storage, ck):
    case = Case(r=4, nt=50, storage=storage, ckpt_every=ck, image_every=4, **SHAPES["small"])
    g = DeviceShot(case)
    g.forward()
    d_obs = case.d_obs(g.nrec)
    img, _ = g.backward_image(d_obs)
    prob = case.oracle_problem()
    fw = prob.forward(keep_u=True)
    bw = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=fw["u"], image_every=4)
    assert rel_l2(img.cpu().numpy(), bw["image"]) <= TOL


@pytest.mark.parametrize("r", [4, 8])
def test_dot_product_on_gpu(r):
    """<F w, q> = <w, F^T q> with the GPU forward data and the GPU source trace
    of the receiver propagation (w is the Ricker wavelet)."""
    import oracle

    case = Case(r=r, nt=60, **SHAPES["small"])
    g = DeviceShot(case)
    data, _ = g.forward()
    q = case.d_obs(g.nrec)
    _, adj = g.backward_image(q, src_adj=True)
    w = oracle.ricker(case.nt, case.dt, case.f0, case.t0)
    lhs = float(np.sum(data.cpu().numpy().astype(np.float64) * q))
    rhs = float(np.dot(w, adj.cpu().numpy().astype(np.float64)))
    assert abs(lhs - rhs) <= TOL * max(abs(lhs), abs(rhs))


def test_source_and_receivers_in_the_sponge():
    extra = np.array([[-3, 4, 5], [31, -2, 3], [5, 6, -4], [0, 0, 25]], np.int32)
    case = Case(r=4, nt=50, src=(-2, 9, 4), extra_rec=extra, **SHAPES["small"])
    g = DeviceShot(case)
    data, _ = g.forward()
    d_obs = case.d_obs(g.nrec)
    img, adj = g.backward_image(d_obs, src_adj=True)
    prob = case.oracle_problem()
    ref = prob.rtm_image(d_obs)
    assert rel_l2(data.cpu().numpy(), ref["data"]) <= TOL
    assert rel_l2(img.cpu().numpy(), ref["image"]) <= TOL
    assert rel_l2(adj.cpu().numpy(), ref["src_adj"]) <= TOL


def test_no_sponge_and_single_step():
    case = Case(r=4, nt=1, nb=0, nx=32, ny=20, nz=12, src=(5, 6, 7))
    g = DeviceShot(case)
    data, last = g.forward(keep_last=True)
    ref = case.oracle_problem().forward(keep_last=True)
    assert rel_l2(last[1].cpu().numpy(), ref["last"][1]) <= TOL
    np.testing.assert_allclose(data.cpu().numpy(), ref["data"], rtol=1e-5, atol=1e-12)


def test_no_receivers():
    import torch

    import paper_1603_03971_gb300 as rtm

    case = Case(r=4, nt=20, **SHAPES["small"])
    p = case.params()
    p.nrec = 0
    ws = rtm.alloc_workspace(p)
    v = torch.from_numpy(case.velocity().astype(np.float32)).cuda()
    c = rtm.model_prep(p, v, ws)
    rec = torch.zeros((0, 3), dtype=torch.int32, device="cuda")
    last = torch.empty((2,) + rtm.padded_shape(p), device="cuda")
    rtm.forward(p, c, rec, ws, data=None, u_last=last)
    rtm.check(ws)
    ref = case.oracle_problem().forward(keep_last=True)
    assert rel_l2(last[1].cpu().numpy(), ref["last"][1]) <= TOL


def test_receiver_out_of_range_is_flagged_not_faulted():
    import paper_1603_03971_gb300 as rtm

    extra = np.array([[500, 0, 0]], np.int32)
    case = Case(r=4, nt=10, extra_rec=extra, **SHAPES["small"])
    g = DeviceShot(case)
    import torch

    data = torch.empty((case.nt, g.nrec), device="cuda")
    rtm.forward(g.p, g.c, g.rec, g.ws, data=data)
    with pytest.raises(rtm.RtmError) as e:
        rtm.check(g.ws)
    assert e.value.code == 1
    rtm.check(g.ws)  # the status word was cleared
    assert float(data[:, -1].abs().max()) == 0.0


def test_cfl_and_bad_models_are_rejected():
    import torch

    import paper_1603_03971_gb300 as rtm
    import oracle

    case = Case(r=4, nt=10, **SHAPES["small"])
    p = case.params()
    ws = rtm.alloc_workspace(p)
    v = torch.full((case.nz, case.ny, case.nx), 1500.0, device="cuda")
    lim = oracle.stability_limit(4)
    v[3, 4, 5] = 1.01 * lim * case.dx / case.dt
    with pytest.raises(rtm.RtmError) as e:
        rtm.model_prep(p, v, ws)
    assert e.value.code == 2
    v[3, 4, 5] = 0.99 * lim * case.dx / case.dt
    rtm.model_prep(p, v, ws)
    v[1, 1, 1] = float("nan")
    with pytest.raises(rtm.RtmError) as e:
        rtm.model_prep(p, v, ws)
    assert e.value.code == 6
    v[1, 1, 1] = -5.0
    with pytest.raises(rtm.RtmError) as e:
        rtm.model_prep(p, v, ws)
    assert e.value.code == 6


@pytest.mark.parametrize("r,storage,ck", [(4, "all", 0), (4, "ckpt", 9), (8, "ckpt", 16)])
def test_gradient_parity(r, storage, ck):
    case = Case(r=r, nt=50, storage=storage, ckpt_every=ck, **SHAPES["small"])
    g = DeviceShot(case, want_grad=True, squared=True)
    g.forward()
    resid = case.d_obs(g.nrec)
    grad = g.grad(resid).cpu().numpy()
    prob = case.oracle_problem(squared=True)
    # hand the oracle the observed data that gives it exactly the same residual
    d_oracle = prob.forward()["data"]
    J, grad_ref = prob.misfit_and_grad(d_oracle - resid)
    assert rel_l2(grad, grad_ref) <= TOL


def test_misfit_kernel():
    import torch

    import paper_1603_03971_gb300 as rtm

    rng = np.random.default_rng(5)
    d = rng.standard_normal((37, 1001)).astype(np.float32)
    o = rng.standard_normal((37, 1001)).astype(np.float32)
    dt, ot = torch.from_numpy(d).cuda(), torch.from_numpy(o).cuda()
    resid = torch.empty_like(dt)
    J, _ = rtm.misfit(dt, ot, resid=resid)
    r64 = d.astype(np.float64) - o.astype(np.float64)
    assert float(J) == pytest.approx(0.5 * float(np.sum(r64 * r64)), rel=1e-9)
    np.testing.assert_array_equal(resid.cpu().numpy(), d - o)


def test_autograd_function_and_central_differences():
    """RtmMisfit: J(v^2) through autograd; its gradient against central
    differences of J on the GPU (relative step 1e-3, FP32 fields)."""
    import torch

    import paper_1603_03971_gb300 as rtm
    import rtm_inputs

    case = Case(r=4, nt=60, storage="ckpt", ckpt_every=16, **SHAPES["small"])
    g = DeviceShot(case, want_grad=True, squared=True)
    p = g.p
    v2 = g.vel.clone()
    blob = rtm_inputs.blob_perturbation(np.sqrt(case.velocity()), 0.05, 4.0) ** 2
    gobs = DeviceShot(case, want_grad=True, vel=blob, squared=True)
    d_obs, _ = gobs.forward()
    x = v2.clone().requires_grad_(True)
    J = rtm.RtmMisfit.apply(x, p, g.rec, d_obs, g.ws)
    J.backward()
    gv = x.grad.double()
    dirs = rtm_inputs.random_directions(v2.shape, 4, seed=9)
    for k, d in enumerate(dirs):
        dt = torch.from_numpy(d / np.abs(d).max()).cuda()
        eps = 1e-3 * float(v2.abs().max())
        Jp = rtm.RtmMisfit.apply(v2 + eps * dt.float(), p, g.rec, d_obs, g.ws)
        Jm = rtm.RtmMisfit.apply(v2 - eps * dt.float(), p, g.rec, d_obs, g.ws)
        fd = float(Jp - Jm) / (2 * eps)
        an = float((gv * dt).sum())
        assert an == pytest.approx(fd, rel=1e-2), (k, an, fd)


def test_shot_host_matches_device_path():
    import torch

    import paper_1603_03971_gb300 as rtm

    case = Case(r=4, nt=40, storage="ckpt", ckpt_every=10, **SHAPES["small"])
    p = case.params()
    rec = case.receivers()
    d_obs = case.d_obs(rec.shape[0]).astype(np.float32)
    v = case.velocity().astype(np.float32)
    ws_h = rtm.alloc_workspace(p, host_io=True)
    img_h = torch.empty((case.nz, case.ny, case.nx), dtype=torch.float32).pin_memory()
    rtm.shot_host(p, torch.from_numpy(v).pin_memory(), torch.from_numpy(rec).pin_memory(),
                  torch.from_numpy(d_obs).pin_memory(), img_h, ws_h)
    g = DeviceShot(case)
    img = torch.zeros((case.nz, case.ny, case.nx), device="cuda")
    rtm.shot(p, g.c, g.rec, torch.from_numpy(d_obs).cuda(), g.ws, img)
    np.testing.assert_array_equal(img_h.numpy(), img.cpu().numpy())
