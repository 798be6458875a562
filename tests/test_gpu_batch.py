"""Batched multi-shot RTM (one persistent cooperative launch per wave) against
the FP64 oracle run shot by shot on each aperture, and invariance of the
result to the wave split and the work-item slab height. Every test runs with
both batched kernels: TMA plane loads (the default) and vector loads."""
import ctypes

import numpy as np
import pytest

import rtm_inputs
from helpers import rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(autouse=True, params=[0, 3, 1], ids=["tma", "tma8", "vector"])
def kernel_variant(request):
    import paper_1603_03971_gb300 as rtm

    for r in (4, 8):
        rtm.set_tuning(r, 0, request.param)
    yield request.param
    for r in (4, 8):
        rtm.set_tuning(r, 0, 0)

FULL = (64, 80, 96)  # nz, ny, nx of the common model
APERTURES = [  # ox, oy, oz, nx, ny, nz, src (x, y, z), rec_z  (aperture coordinates)
    (0, 0, 0, 40, 32, 32, (20, 16, 3), 2),
    (30, 20, 0, 56, 48, 48, (28, 24, 4), 2),
    (10, 40, 8, 32, 36, 40, (5, 30, 6), 1),
]


def _apertures():
    from paper_1603_03971_gb300 import batch

    return [batch.Aperture(ox, oy, oz, nx, ny, nz, *src, rec_z)
            for ox, oy, oz, nx, ny, nz, src, rec_z in APERTURES]


def _setup(r, nt, k, ie, nb=8):
    import paper_1603_03971_gb300 as rtm

    nz, ny, nx = FULL
    vel = rtm_inputs.smooth_random_velocity(nx, ny, nz, 4.0, 1500.0, 3000.0, seed=21)
    dt = rtm_inputs.courant_dt(10.0, 3000.0)
    p = rtm.make_params(nx, ny, nz, nb, r, nt, 10.0, dt, 25.0, 0.04, (0, 0, 0), 0,
                        storage="ckpt", ckpt_every=k, image_every=ie)
    dobs = [rtm_inputs.standard_normal((nt, a[4], a[3]), seed=30 + i) * 1e-3
            for i, a in enumerate(APERTURES)]
    return p, vel, dobs


def _oracle(p, vel, dobs):
    import oracle

    nz, ny, nx = FULL
    image = np.zeros((nz, ny, nx))
    datas = []
    for (ox, oy, oz, anx, any_, anz, src, rec_z), d in zip(APERTURES, dobs):
        v = vel[oz:oz + anz, oy:oy + any_, ox:ox + anx]
        rec = rtm_inputs.surface_receivers(anx, any_, rec_z)
        prob = oracle.Problem(v, p.nb, p.radius, p.dx, p.dt, p.nt, p.f0, p.t0, src, rec)
        fw = prob.forward(keep_u=True)
        bw = prob.grid.adjoint(prob.w, prob.src, prob.rec, d.reshape(p.nt, -1), snap_u=fw["u"],
                               image_every=p.image_every)
        image[oz:oz + anz, oy:oy + any_, ox:ox + anx] += bw["image"]
        datas.append(fw["data"].reshape(p.nt, any_, anx))
    return image, datas


def _run(p, vel, dobs, budget=0, zchunk=0):
    import torch

    from paper_1603_03971_gb300 import batch

    aps = _apertures()
    v = torch.from_numpy(vel.astype(np.float32)).cuda()
    d = torch.from_numpy(np.concatenate([x.ravel() for x in dobs]).astype(np.float32)).cuda()
    data = torch.zeros_like(d)
    img = torch.zeros(FULL, device="cuda")
    ws = batch.alloc_workspace(p, aps, budget)
    batch.run(p, aps, v, d, img, ws, data=data, budget=budget, zchunk=zchunk)
    import paper_1603_03971_gb300 as rtm

    rtm.check(ws)
    return img.cpu().numpy(), data.cpu().numpy()


@pytest.mark.parametrize("r,nt,k,ie", [(4, 40, 12, 1), (8, 36, 10, 2)])
def test_batch_matches_oracle_per_shot(r, nt, k, ie):
    p, vel, dobs = _setup(r, nt, k, ie)
    img, data = _run(p, vel, dobs)
    ref_img, ref_data = _oracle(p, vel, dobs)
    assert rel_l2(img, ref_img) <= TOL
    off = 0
    for rd in ref_data:
        n = rd.size
        assert rel_l2(data[off:off + n].reshape(rd.shape), rd) <= TOL
        off += n


def test_batch_is_independent_of_waves_and_slabs():
    p, vel, dobs = _setup(4, 30, 8, 1)
    img1, data1 = _run(p, vel, dobs)
    img2, data2 = _run(p, vel, dobs, budget=1)  # one shot per wave
    img3, data3 = _run(p, vel, dobs, zchunk=16)
    np.testing.assert_array_equal(img1, img2)
    np.testing.assert_array_equal(img1, img3)
    np.testing.assert_array_equal(data1, data3)


def test_batch_rejects_bad_apertures_on_the_host():
    import paper_1603_03971_gb300 as rtm
    from paper_1603_03971_gb300 import _lib, batch

    p, _, _ = _setup(4, 10, 4, 1)
    bad = [batch.Aperture(90, 0, 0, 40, 32, 32, 1, 1, 1, 1)]  # beyond the model in x
    arr = (batch.Aperture * 1)(*bad)
    assert _lib.lib().rtm_batch_workspace_size(ctypes.byref(p), 1, arr, 0) == 0
    del rtm


def test_batch_wait_timeout_is_reported_not_hung():
    """A host-injected wait that nothing completes runs out after about a
    second: rtm_batch returns RTM_ERR_TIMEOUT, the device stays usable and
    the next batch is correct."""
    import time

    import paper_1603_03971_gb300 as rtm
    from paper_1603_03971_gb300 import batch

    p, vel, dobs = _setup(4, 12, 6, 1)
    batch.set_wait(1.0, poison_shot=1)
    try:
        t0 = time.time()
        with pytest.raises(rtm.RtmError) as e:
            _run(p, vel, dobs)
        assert e.value.code == 5
        assert time.time() - t0 < 60
    finally:
        batch.set_wait(20.0, -1)
    img, _ = _run(p, vel, dobs)
    ref, _ = _oracle(p, vel, dobs)
    assert rel_l2(img, ref) <= TOL


def test_batch_at_full_size_matches_single_shots():
    """The batched-shots workload at its full size (1024 x 1024 x 512 layered
    / salt model, radius 8, apertures from 128 x 128 x 256 upward): four of
    its seeded apertures, 60 steps, checkpoints every 10. The oracle cannot
    run these sizes; the single-shot path, checked against the oracle on
    every shape class, is the reference: the batched image equals the sum of
    the single-shot images of the same apertures and data within the
    wavefield tolerance (the two paths form their FP32 sums in different
    orders)."""
    import torch

    import paper_1603_03971_gb300 as rtm
    from paper_1603_03971_gb300 import batch

    cfg = rtm_inputs.BATCH_WORKLOAD
    nz, ny, nx = cfg["model_shape"]
    nt, nb, r = 60, cfg["nb"], cfg["radius"]
    vel_np = rtm_inputs.layered_salt_velocity(nx, ny, nz, seed=cfg["seed"])
    vel = torch.from_numpy(vel_np).cuda()
    origin, size = rtm_inputs.batch_apertures(cfg["nshots"], (nz, ny, nx), seed=cfg["seed"])
    pick = [0, 1, 2, 3]
    aps = [batch.Aperture(int(origin[i][0]), int(origin[i][1]), int(origin[i][2]), int(size[i][0]),
                          int(size[i][1]), int(size[i][2]), int(size[i][0]) // 2,
                          int(size[i][1]) // 2, 4, 2) for i in pick]
    dt = rtm_inputs.courant_dt(cfg["dx"], cfg["vmax"])
    p = rtm.make_params(nx, ny, nz, nb, r, nt, cfg["dx"], dt, cfg["f0"], 1.0 / cfg["f0"],
                        (0, 0, 0), 0, storage="ckpt", ckpt_every=10)
    dobs = [rtm_inputs.standard_normal((nt, a.ny, a.nx), seed=90 + i).astype(np.float32) * 1e-3
            for i, a in enumerate(aps)]
    d = torch.from_numpy(np.concatenate([x.ravel() for x in dobs])).cuda()
    img = torch.zeros((nz, ny, nx), device="cuda")
    ws = batch.alloc_workspace(p, aps)
    batch.run(p, aps, vel, d, img, ws)
    rtm.check(ws)
    del ws
    ref = torch.zeros_like(img)
    for a, dd in zip(aps, dobs):
        q = rtm.make_params(a.nx, a.ny, a.nz, nb, r, nt, cfg["dx"], dt, cfg["f0"],
                            1.0 / cfg["f0"], (a.src_x, a.src_y, a.src_z), a.nx * a.ny,
                            storage="ckpt", ckpt_every=10)
        w = rtm.alloc_workspace(q)
        v = vel[a.oz:a.oz + a.nz, a.oy:a.oy + a.ny, a.ox:a.ox + a.nx].contiguous()
        c = rtm.model_prep(q, v, w)
        rec = torch.from_numpy(rtm_inputs.surface_receivers(a.nx, a.ny, a.rec_z)).cuda()
        im = torch.zeros((a.nz, a.ny, a.nx), device="cuda")
        rtm.shot(q, c, rec, torch.from_numpy(dd.reshape(nt, -1)).cuda(), w, im)
        rtm.check(w)
        ref[a.oz:a.oz + a.nz, a.oy:a.oy + a.ny, a.ox:a.ox + a.nx] += im
        del w
    assert float(ref.abs().max()) > 0
    assert rel_l2(img.cpu().numpy(), ref.cpu().numpy()) <= TOL


_FULL_ORACLE = {}


def test_batch_at_full_size_matches_the_oracle_on_real_apertures():
    """The batched-shots workload at its full size, in its launch
    configuration: all 32 seeded apertures of the 1024 x 1024 x 512 layered /
    salt model in one batch (radius 8, checkpoints every 10, 30 steps), and
    two of its real apertures (160 x 160 x 288 and 160 x 256 x 288) against
    the FP64 oracle run on each whole aperture: at radius 8 the stencil's
    reach after 30 steps (240 cells) spans the aperture, so the exact crop is
    the aperture itself. The modelled data of those two shots are compared
    directly; the other shots get zero observed data, so the image is the
    sum of the two shots' images."""
    import torch

    import oracle
    import paper_1603_03971_gb300 as rtm
    from paper_1603_03971_gb300 import batch

    cfg = rtm_inputs.BATCH_WORKLOAD
    nz, ny, nx = cfg["model_shape"]
    nt, k, nb, r = 30, 10, cfg["nb"], cfg["radius"]
    vel_np = rtm_inputs.layered_salt_velocity(nx, ny, nz, seed=cfg["seed"])
    origin, size = rtm_inputs.batch_apertures(cfg["nshots"], (nz, ny, nx), seed=cfg["seed"])
    aps = [batch.Aperture(int(o[0]), int(o[1]), int(o[2]), int(s[0]), int(s[1]), int(s[2]),
                          int(s[0]) // 2, int(s[1]) // 2, 4, 2) for o, s in zip(origin, size)]
    picked = [15, 18]
    dt = rtm_inputs.courant_dt(cfg["dx"], cfg["vmax"])
    p = rtm.make_params(nx, ny, nz, nb, r, nt, cfg["dx"], dt, cfg["f0"], 1.0 / cfg["f0"],
                        (0, 0, 0), 0, storage="ckpt", ckpt_every=k)
    dobs = [rtm_inputs.standard_normal((nt, a.ny, a.nx), seed=120 + i).astype(np.float32) * 1e-3
            if i in picked else np.zeros((nt, a.ny, a.nx), np.float32)
            for i, a in enumerate(aps)]
    vel = torch.from_numpy(vel_np).cuda()
    d = torch.from_numpy(np.concatenate([x.ravel() for x in dobs])).cuda()
    data = torch.zeros_like(d)
    img = torch.zeros((nz, ny, nx), device="cuda")
    ws = batch.alloc_workspace(p, aps)
    batch.run(p, aps, vel, d, img, ws, data=data)
    rtm.check(ws)
    del ws
    offs = np.cumsum([0] + [nt * a.nx * a.ny for a in aps])
    data_np = data.cpu().numpy()
    if not _FULL_ORACLE:
        for i in picked:
            a = aps[i]
            v = vel_np[a.oz:a.oz + a.nz, a.oy:a.oy + a.ny, a.ox:a.ox + a.nx].astype(np.float64)
            rec = rtm_inputs.surface_receivers(a.nx, a.ny, a.rec_z)
            prob = oracle.Problem(v, nb, r, cfg["dx"], dt, nt, cfg["f0"], 1.0 / cfg["f0"],
                                  (a.src_x, a.src_y, a.src_z), rec)
            fw = prob.forward(keep_u=True)
            bw = prob.grid.adjoint(prob.w, prob.src, prob.rec,
                                   dobs[i].reshape(nt, -1).astype(np.float64), snap_u=fw["u"])
            _FULL_ORACLE[i] = (fw["data"], bw["image"])
            del fw, bw, prob
    ref_img = {}
    for i in picked:
        a = aps[i]
        ref_data, img_i = _FULL_ORACLE[i]
        got = data_np[offs[i]:offs[i + 1]].reshape(nt, -1)
        assert rel_l2(got, ref_data) <= TOL, i
        ref_img[i] = img_i
    # the image: the two shots' images summed over their (overlapping) apertures
    boxes = [(aps[i], ref_img[i]) for i in picked]
    z0 = min(a.oz for a, _ in boxes)
    z1 = max(a.oz + a.nz for a, _ in boxes)
    y0 = min(a.oy for a, _ in boxes)
    y1 = max(a.oy + a.ny for a, _ in boxes)
    x0 = min(a.ox for a, _ in boxes)
    x1 = max(a.ox + a.nx for a, _ in boxes)
    ref = np.zeros((z1 - z0, y1 - y0, x1 - x0))
    for a, im in boxes:
        ref[a.oz - z0:a.oz - z0 + a.nz, a.oy - y0:a.oy - y0 + a.ny,
            a.ox - x0:a.ox - x0 + a.nx] += im
    got = img[z0:z1, y0:y1, x0:x1].cpu().numpy()
    assert np.abs(ref).max() > 0
    assert rel_l2(got, ref) <= TOL
    # nothing outside the two apertures
    tot = float(img.abs().sum())
    assert tot == pytest.approx(float(np.abs(got).sum()), rel=1e-6)
