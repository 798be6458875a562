"""Imaging-condition variants on the GPU against the oracle: the source
illumination accumulated during receiver propagation (store-all, checkpoint
and learned storage), the illumination-normalised image and the
Laplacian-filtered image."""
import numpy as np
import pytest

import rtm_inputs
from helpers import Case, DeviceShot, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-4

SMALL = dict(nx=28, ny=24, nz=20, nb=6)
RAGGED = dict(nx=100, ny=44, nz=37, nb=10)


def _illum_run(g, d_obs, ae_params=None):
    import torch

    rd = torch.from_numpy(np.ascontiguousarray(d_obs, dtype=np.float32)).cuda()
    img = torch.zeros((g.p.nz, g.p.ny, g.p.nx), device="cuda")
    illum = torch.zeros_like(img)
    g.rtm.backward_image_illum(g.p, g.c, g.rec, rd, g.ws, img, illum, ae_params=ae_params)
    g.rtm.check(g.ws)
    return img, illum


@pytest.mark.parametrize("r,storage,ck,ie,shape", [
    (4, "all", 0, 1, SMALL), (4, "ckpt", 9, 2, SMALL), (8, "ckpt", 16, 3, RAGGED),
    (4, "ckpt", 7, 1, dict(nx=32, ny=24, nz=20, nb=8))])  # last: 16-byte vector path
def test_illumination_matches_oracle(r, storage, ck, ie, shape):
    from oracle import imaging

    case = Case(r=r, nt=48, storage=storage, ckpt_every=ck, image_every=ie, **shape)
    g = DeviceShot(case)
    g.forward()
    d_obs = case.d_obs(g.nrec)
    img, illum = _illum_run(g, d_obs)
    prob = case.oracle_problem()
    fw = prob.forward(keep_u=True)
    bw = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=fw["u"], image_every=ie)
    assert rel_l2(img.cpu().numpy(), bw["image"]) <= TOL
    assert rel_l2(illum.cpu().numpy(), imaging.illumination(fw["u"], ie)) <= TOL
    # the image is the one the plain imaging call gives (the backward pass
    # consumes the checkpoints in place, so the forward pass runs again)
    g.forward()
    plain, _ = g.backward_image(d_obs)
    assert bool((plain == img).all())


def test_illumination_in_learned_storage_is_that_of_the_decoded_snapshots():
    """With learned storage the illumination uses the decoded snapshots, as
    the image does: it equals the oracle's illumination of the oracle
    codec's reconstruction of the same latents within the codec tolerance."""
    import torch

    from oracle import ae as oae
    from oracle import imaging
    import paper_1603_03971_gb300 as rtm

    ie = 4
    case = Case(r=4, nt=40, storage="learned", image_every=ie, nx=32, ny=24, nz=20, nb=6)
    P = rtm_inputs.ae_flat(rtm_inputs.ae_init_params(2)).astype(np.float32)
    Pd = torch.from_numpy(P).cuda()
    g = DeviceShot(case)
    rtm.forward_learned(g.p, g.c, g.rec, Pd, g.ws)
    rtm.check(g.ws)
    d_obs = case.d_obs(g.nrec)
    _, illum = _illum_run(g, d_obs, ae_params=Pd)
    # oracle: snapshots from the oracle propagator, coded and decoded by the oracle codec
    fw = case.oracle_problem().forward(keep_u=True)
    params = oae.unflatten(P.astype(np.float64))
    rec_snaps = np.zeros_like(fw["u"])
    for m in range(ie, case.nt + 1, ie):
        lat, sc = oae.encode(params, fw["u"][m - 1].astype(np.float32).astype(np.float64))
        rec_snaps[m - 1] = oae.decode(params, lat, sc)
    # quadratic in the decoded snapshots: twice the codec tolerance
    assert rel_l2(illum.cpu().numpy(), imaging.illumination(rec_snaps, ie)) <= 4e-3


@pytest.mark.parametrize("r,shape", [(4, (20, 24, 28)), (8, (9, 30, 17)), (4, (3, 2, 5))])
def test_image_filter_matches_oracle(r, shape):
    import torch

    from oracle import imaging
    import paper_1603_03971_gb300 as rtm

    nz, ny, nx = shape
    p = rtm.make_params(nx, ny, nz, 4, r, 10, 7.5, 1e-4, 20.0, 0.05, (0, 0, 0), 0)
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")  # the status block is enough
    image = rtm_inputs.standard_normal(shape, 71, np.float32)
    illum = (rtm_inputs.standard_normal(shape, 72, np.float32) ** 2).astype(np.float32)
    It, Lt = torch.from_numpy(image).cuda(), torch.from_numpy(illum).cuda()
    norm, lap = rtm.image_filter(p, It, ws, illum=Lt, eps_rel=1e-2)
    rtm.check(ws)
    ref_n = imaging.normalized_image(image.astype(np.float64), illum.astype(np.float64), 1e-2)
    ref_l = imaging.laplacian_filter(image.astype(np.float64), r, 7.5)
    assert rel_l2(norm.cpu().numpy(), ref_n) <= 1e-6
    assert rel_l2(lap.cpu().numpy(), ref_l) <= 1e-6
    only_lap = rtm.image_filter(p, It, ws, normalized=False)
    assert only_lap[0] is None and torch.equal(only_lap[1], lap)


def test_image_filter_rejects_bad_arguments():
    import torch

    import paper_1603_03971_gb300 as rtm

    p = rtm.make_params(8, 8, 8, 4, 4, 10, 10.0, 1e-4, 20.0, 0.05, (0, 0, 0), 0)
    ws = rtm.alloc_workspace(p)
    img = torch.zeros((8, 8, 8), device="cuda")
    with pytest.raises(rtm.RtmError):
        rtm.image_filter(p, img, ws, illum=None)  # normalisation without illumination
    with pytest.raises(rtm.RtmError):
        rtm.image_filter(p, img, ws, illum=img, eps_rel=0.0)
