"""Off-grid source and receivers (Kaiser-windowed sinc tap tables) on the GPU:

* on-grid positions through the off-grid calls reproduce the on-grid calls
  bit for bit (single taps of weight 1, the same arithmetic);
* positions between grid points match the FP64 oracle's distributed
  injection and gather (wavefield tolerance), through checkpointed and
  boundary storage;
* the two-layer 64^3 workload with its source and receivers moved off the
  grid: data and image against the oracle."""
import numpy as np
import pytest

import rtm_inputs
from helpers import Case, DeviceShot, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _taps(g, src_xyz, rec_xyz):
    import paper_1603_03971_gb300 as rtm

    return rtm.offgrid_taps(g.p, src_xyz, rec_xyz, device="cuda")


@pytest.mark.parametrize("r", [4, 8])
def test_on_grid_points_equal_the_on_grid_calls(r):
    import torch

    import paper_1603_03971_gb300 as rtm

    case = Case(r=r, nt=40, storage="ckpt", ckpt_every=9)
    g = DeviceShot(case)
    data_ref, _ = g.forward()
    d_obs = case.d_obs(g.nrec)
    img_ref, _ = g.backward_image(d_obs)
    taps = _taps(g, np.array(case.src, np.float64), g.rec_np.astype(np.float64))
    data = torch.empty_like(data_ref)
    rtm.forward_offgrid(g.p, g.c, taps, g.ws, data=data)
    rtm.check(g.ws)
    assert torch.equal(data, data_ref)
    img = torch.zeros_like(img_ref)
    rtm.shot_offgrid(g.p, g.c, taps, torch.from_numpy(d_obs.astype(np.float32)).cuda(), g.ws,
                     img)
    rtm.check(g.ws)
    assert torch.equal(img, img_ref)


def _oracle(case, src_xyz, rec_xyz, d_obs, image_every=1):
    from oracle import offgrid

    prob = case.oracle_problem()
    shape = prob.grid.shape
    src = offgrid.point_taps(src_xyz, case.nb, shape)
    recs = offgrid.taps_of(rec_xyz, case.nb, shape)
    fw = offgrid.forward(prob.grid, prob.w, src, recs, keep_u=True)
    bw = offgrid.adjoint(prob.grid, recs, d_obs, snap_u=fw["u"], image_every=image_every)
    return fw["data"], bw["image"]


@pytest.mark.parametrize("r,storage", [(4, "ckpt"), (8, "ckpt"), (4, "boundary")])
def test_off_grid_shot_matches_the_oracle(r, storage):
    import torch

    import paper_1603_03971_gb300 as rtm

    case = Case(nx=36, ny=28, nz=30, nb=8, r=r, nt=50, storage=storage, ckpt_every=12,
                src=(17, 13, 4))
    g = DeviceShot(case)
    src = np.array([17.35, 13.6, 4.45])
    rng = np.random.default_rng(8)
    rec = np.column_stack([rng.uniform(1.0, case.nx - 2.0, 40), rng.uniform(1.0, case.ny - 2.0, 40),
                           np.full(40, 2.5)])
    rec[:6, 2] = 2.0  # some receivers on the grid in z only
    p = g.p.copy(nrec=len(rec))
    taps = rtm.offgrid_taps(p, src, rec, device="cuda")
    ws = rtm.alloc_workspace(p)
    d_obs = rtm_inputs.standard_normal((case.nt, len(rec)), seed=9) * 1e-3
    data = torch.empty((case.nt, len(rec)), device="cuda")
    img = torch.zeros((case.nz, case.ny, case.nx), device="cuda")
    rtm.shot_offgrid(p, g.c, taps, torch.from_numpy(d_obs.astype(np.float32)).cuda(), ws, img,
                     data=data)
    rtm.check(ws)
    ref_data, ref_img = _oracle(case, src, rec, d_obs)
    assert rel_l2(data.cpu().numpy(), ref_data) <= TOL
    assert rel_l2(img.cpu().numpy(), ref_img) <= TOL


def test_two_layer_64_off_grid_against_the_oracle():
    """The two-layer 64^3 workload (104^3 padded, 300 steps, every snapshot
    stored) with its source at (32.4, 31.7, 4.5) and its 64 x 64 receivers
    half a cell off the grid in x, y and z (512 taps each)."""
    import torch

    import oracle
    import paper_1603_03971_gb300 as rtm
    from oracle import offgrid

    w = rtm_inputs.WORKLOADS["two_layer_64"]
    v = w.velocity_model()
    src = np.array([32.4, 31.7, 4.5])
    xs, ys = np.meshgrid(np.arange(w.nx) + 0.5, np.arange(w.ny) + 0.5, indexing="xy")
    rec = np.column_stack([xs.ravel(), ys.ravel(), np.full(xs.size, 2.5)])
    rec = rec[(rec[:, 0] < w.nx - 1) & (rec[:, 1] < w.ny - 1)]
    p = rtm.params_for(w, nrec=len(rec))
    ws = rtm.alloc_workspace(p)
    c = rtm.model_prep(p, torch.from_numpy(v).float().cuda(), ws)
    taps = rtm.offgrid_taps(p, src, rec, device="cuda")
    prob = oracle.Problem(v, w.nb, w.radius, w.dx, w.dt, w.nt, w.f0, w.t0, w.src,
                          w.receivers()[:1])
    shape = prob.grid.shape
    st = offgrid.point_taps(src, w.nb, shape)
    rt = offgrid.taps_of(rec, w.nb, shape)
    fw = offgrid.forward(prob.grid, prob.w, st, rt, keep_u=True)
    d_obs = fw["data"]
    img_ref = offgrid.adjoint(prob.grid, rt, d_obs, snap_u=fw["u"])["image"]
    data = torch.empty((w.nt, len(rec)), device="cuda")
    img = torch.zeros((w.nz, w.ny, w.nx), device="cuda")
    rtm.shot_offgrid(p, c, taps, torch.from_numpy(d_obs.astype(np.float32)).cuda(), ws, img,
                     data=data)
    rtm.check(ws)
    assert rel_l2(data.cpu().numpy(), d_obs) <= TOL
    assert rel_l2(img.cpu().numpy(), img_ref) <= TOL


def test_points_outside_the_grid_are_rejected_on_the_host():
    import paper_1603_03971_gb300 as rtm

    p = Case().params()
    with pytest.raises(rtm.RtmError):
        rtm.offgrid_taps(p, (100.5, 1.0, 1.0), np.zeros((p.nrec, 3)))
