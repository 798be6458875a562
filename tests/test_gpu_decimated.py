"""Decimated storage (the non-learned 8x scheme beside learned storage):
every other model sample per axis of each imaging snapshot kept in float32,
rebuilt by linear interpolation before the imaging step.

Parity: the GPU shot against the oracle chain (FP64 propagation, the
oracle's decimation and interpolation of each snapshot, FP64 receiver
propagation and imaging). The kept samples are exact float32 copies and the
interpolation weights (1, 1/2, 1/4, 1/8) are exact, so the bar is the
wavefield tolerance, 1e-4."""
import numpy as np
import pytest

from helpers import Case, DeviceShot, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _decimated_image(case, g, d_obs_np, window=0):
    import torch

    import paper_1603_03971_gb300 as rtm

    pd = case.params()
    pd.storage = rtm.RTM_STORE_DECIMATED
    pd.ckpt_every = window
    wd = rtm.alloc_workspace(pd)
    dobs = torch.from_numpy(np.ascontiguousarray(d_obs_np, dtype=np.float32)).cuda()
    img = torch.zeros((case.nz, case.ny, case.nx), device="cuda")
    data = torch.empty((case.nt, g.nrec), device="cuda")
    rtm.shot(pd, g.c, g.rec, dobs, wd, img, data=data)
    rtm.check(wd)
    return img.cpu().numpy().astype(np.float64), data.cpu().numpy()


@pytest.mark.parametrize("r", [4, 8])
@pytest.mark.parametrize("window,shape,nb", [(0, (32, 28, 24), 8), (13, (32, 28, 24), 8),
                                             (0, (38, 21, 27), 9), (9, (100, 44, 37), 8)])
def test_decimated_shot_matches_the_oracle_chain(r, window, shape, nb):
    """Even and odd model sides (x is even: padded rows are 16-byte aligned);
    the largest shape spans several stencil tiles with ragged tails."""
    from oracle import ae as oae

    nx, ny, nz = shape
    ie = 4
    case = Case(nx=nx, ny=ny, nz=nz, nb=nb, r=r, nt=40, image_every=ie,
                src=(nx // 2, ny // 2, 3))
    g = DeviceShot(case)
    d_obs = case.d_obs(g.nrec)
    img, data = _decimated_image(case, g, d_obs, window)
    prob = case.oracle_problem()
    fw = prob.forward(keep_u=True)
    assert rel_l2(data, fw["data"]) <= TOL
    su = np.zeros_like(fw["u"])
    for m in range(ie, case.nt + 1, ie):
        u = fw["u"][m - 1]
        su[m - 1] = u if m <= window else oae.trilinear_upsample(oae.decimate(u), u.shape)
    ref = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=su,
                            image_every=ie)["image"]
    assert rel_l2(img, ref) <= TOL


def test_exact_window_over_the_whole_run_is_the_store_all_image():
    case = Case(nx=32, ny=28, nz=24, nb=8, r=4, nt=40, image_every=4)
    g = DeviceShot(case)
    d_obs = case.d_obs(g.nrec)
    img, _ = _decimated_image(case, g, d_obs, window=case.nt)
    g.forward()
    ref = g.backward_image(d_obs)[0].cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(img, ref)


def test_decimated_workspace_is_an_eighth_of_the_snapshots():
    import paper_1603_03971_gb300 as rtm

    case = Case(nx=64, ny=64, nz=64, nb=8, r=4, nt=400, image_every=4)
    pa = case.params()
    pd = case.params()
    pd.storage = rtm.RTM_STORE_DECIMATED
    n_snap = case.nt // 4
    grow = rtm.workspace_size(pd) - rtm.workspace_size(pd.copy(nt=4))
    # every imaging step adds one float32 coarse snapshot, 32^3 * 4 bytes
    # (and the wavelet table grows by nt floats)
    coarse = (n_snap - 1) * 32 ** 3 * 4
    assert coarse <= grow <= coarse + 4096
    grow_all = rtm.workspace_size(pa) - rtm.workspace_size(pa.copy(nt=4))
    assert grow_all >= 8 * coarse
