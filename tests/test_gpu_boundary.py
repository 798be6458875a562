"""Boundary storage on the GPU: the forward pass keeps the model region's
boundary band of every state, the backward pass recovers the source field by
reverse time stepping and images it. The image matches the oracle's and the
store-all image (FP32 reverse stepping adds rounding only), the source trace
is unchanged, and the edge cases (few steps, source in the band or in the
sponge, thin models, ragged tiles) hold."""
import numpy as np
import pytest

from helpers import Case, DeviceShot, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-4
SMALL = dict(nx=28, ny=24, nz=20, nb=6)
RAGGED = dict(nx=30, ny=26, nz=23, nb=5)  # nb % 4 != 0: the model starts inside a vector
THIN = dict(nx=10, ny=10, nz=11, nb=7, src=(5, 5, 5))  # 2 x 2 x 3 inner cells at r = 4


@pytest.fixture(autouse=True)
def _reset_tuning():
    import paper_1603_03971_gb300 as rtm

    yield
    rtm.set_tuning(4, 0, 0)
    rtm.set_tuning(8, 0, 0)


def _image(case, d_obs=None):
    g = DeviceShot(case)
    g.forward()
    if d_obs is None:
        d_obs = case.d_obs(g.nrec)
    img, adj = g.backward_image(d_obs, src_adj=True)
    return g, d_obs, img.cpu().numpy().astype(np.float64), adj.cpu().numpy()


@pytest.mark.parametrize("variant", [2, 3, 1])
@pytest.mark.parametrize("r,ie,nt,shape", [
    (4, 1, 60, SMALL), (4, 3, 61, RAGGED), (8, 1, 50, dict(nx=36, ny=34, nz=35, nb=8)),
    (8, 2, 44, RAGGED), (4, 1, 40, THIN)])
def test_boundary_image_matches_oracle_and_store_all(variant, r, ie, nt, shape):
    import paper_1603_03971_gb300 as rtm

    rtm.set_tuning(r, 0, variant)
    base = dict(r=r, nt=nt, image_every=ie, **shape)
    cb = Case(storage="boundary", **base)
    gb, d_obs, img_b, adj_b = _image(cb)
    ca = Case(storage="all", **base)
    _, _, img_a, adj_a = _image(ca, d_obs)
    prob = cb.oracle_problem()
    fw = prob.forward(keep_u=True)
    bw = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=fw["u"], image_every=ie)
    assert rel_l2(img_b, bw["image"]) <= TOL
    assert rel_l2(img_b, img_a) <= 2e-5
    # the receiver field does not depend on the storage
    assert np.array_equal(adj_b, adj_a)


@pytest.mark.parametrize("nt", [1, 2, 3, 4])
def test_few_steps(nt):
    base = dict(r=4, nt=nt, **SMALL)
    cb = Case(storage="boundary", **base)
    _, d_obs, img_b, _ = _image(cb)
    _, _, img_a, _ = _image(Case(storage="all", **base), d_obs)
    assert rel_l2(img_b, img_a) <= 1e-6


@pytest.mark.parametrize("src", [(14, 12, 1), (-3, 12, 9), (14, 12, 10)])
def test_source_in_band_sponge_and_interior(src):
    base = dict(r=4, nt=50, src=src, **SMALL)
    cb = Case(storage="boundary", **base)
    _, d_obs, img_b, _ = _image(cb)
    prob = cb.oracle_problem()
    fw = prob.forward(keep_u=True)
    ref = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=fw["u"])["image"]
    assert rel_l2(img_b, ref) <= TOL


def test_shot_and_illumination():
    import torch

    from oracle import imaging
    import paper_1603_03971_gb300 as rtm

    case = Case(storage="boundary", r=4, nt=48, image_every=2, **SMALL)
    g = DeviceShot(case)
    d_obs = case.d_obs(g.nrec)
    dd = torch.from_numpy(np.ascontiguousarray(d_obs, dtype=np.float32)).cuda()
    img = torch.zeros((case.nz, case.ny, case.nx), device="cuda")
    rtm.shot(g.p, g.c, g.rec, dd, g.ws, img)
    rtm.check(g.ws)
    prob = case.oracle_problem()
    fw = prob.forward(keep_u=True)
    ref = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=fw["u"], image_every=2)
    assert rel_l2(img.cpu().numpy(), ref["image"]) <= TOL
    g.forward()
    img2 = torch.zeros_like(img)
    illum = torch.zeros_like(img)
    rtm.backward_image_illum(g.p, g.c, g.rec, dd, g.ws, img2, illum)
    rtm.check(g.ws)
    assert rel_l2(img2.cpu().numpy(), ref["image"]) <= TOL
    assert rel_l2(illum.cpu().numpy(), imaging.illumination(fw["u"], 2)) <= TOL


def test_long_run_reverse_error_stays_small():
    """400 steps of FP32 reverse stepping: the image stays within 1e-5 of the
    store-all image on the same device."""
    base = dict(r=4, nt=400, nx=48, ny=44, nz=40, nb=8, src=(24, 22, 4))
    cb = Case(storage="boundary", **base)
    _, d_obs, img_b, _ = _image(cb)
    _, _, img_a, _ = _image(Case(storage="all", **base), d_obs)
    assert rel_l2(img_b, img_a) <= 1e-5
