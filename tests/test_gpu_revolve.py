"""Binomial checkpointing on the GPU: the image and source trace equal the
store-all ones bit for bit (the same kernels recompute the same fields) and
match the oracle, for zero to many slots and imaging every k steps."""
import numpy as np
import pytest

from helpers import Case, DeviceShot, rel_l2

pytestmark = pytest.mark.gpu
SMALL = dict(nx=28, ny=24, nz=20, nb=6)
RAGGED = dict(nx=100, ny=44, nz=37, nb=10)


@pytest.mark.parametrize("slots,ie,nt,r,shape", [
    (0, 1, 12, 4, SMALL), (2, 1, 40, 4, SMALL), (3, 2, 50, 4, SMALL), (1, 3, 47, 8, RAGGED),
    (8, 1, 40, 4, SMALL), (40, 1, 30, 4, SMALL)])
def test_revolve_equals_store_all_and_the_oracle(slots, ie, nt, r, shape):
    import torch

    base = dict(r=r, nt=nt, image_every=ie, **shape)
    ca = Case(storage="all", **base)
    ga = DeviceShot(ca)
    ga.forward()
    d_obs = ca.d_obs(ga.nrec)
    img_a, adj_a = ga.backward_image(d_obs, src_adj=True)
    cr = Case(storage="revolve", ckpt_every=slots, **base)
    gr = DeviceShot(cr)
    gr.forward()
    img_r, adj_r = gr.backward_image(d_obs, src_adj=True)
    assert torch.equal(img_r, img_a)
    assert torch.equal(adj_r, adj_a)
    prob = ca.oracle_problem()
    fw = prob.forward(keep_u=True)
    bw = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=fw["u"], image_every=ie)
    assert rel_l2(img_r.cpu().numpy(), bw["image"]) <= 1e-4


def test_revolve_shot_and_workspace():
    """rtm_shot with binomial checkpointing gives the store-all image; its
    workspace holds the slots and one snapshot, independent of nt."""
    import torch

    import paper_1603_03971_gb300 as rtm

    base = dict(r=4, nt=60, image_every=1, **SMALL)
    ca = Case(storage="all", **base)
    ga = DeviceShot(ca)
    d_obs = ca.d_obs(ga.nrec)
    dd = torch.from_numpy(np.ascontiguousarray(d_obs, dtype=np.float32)).cuda()
    img_a = torch.zeros((ca.nz, ca.ny, ca.nx), device="cuda")
    rtm.shot(ga.p, ga.c, ga.rec, dd, ga.ws, img_a)
    cr = Case(storage="revolve", ckpt_every=4, **base)
    gr = DeviceShot(cr)
    img_r = torch.zeros_like(img_a)
    rtm.shot(gr.p, gr.c, gr.rec, dd, gr.ws, img_r)
    rtm.check(gr.ws)
    assert torch.equal(img_r, img_a)
    p_long = cr.params()
    p_long.nt = 600
    assert rtm.workspace_size(p_long) - rtm.workspace_size(cr.params()) < 4 * 600 + 4096
