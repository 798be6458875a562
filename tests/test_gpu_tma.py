"""The TMA plane-load variant of the stencil (tuning variant 2): the same
oracle parity as the vector-load variant, over shapes with ragged tiles and
z slabs shorter than the stencil radius, in all five kernel modes."""
import numpy as np
import pytest

from helpers import Case, DeviceShot, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-4
SHAPES = {
    "small": dict(nx=28, ny=24, nz=20, nb=6),
    "ragged": dict(nx=100, ny=44, nz=37, nb=10),
    "thin": dict(nx=4, ny=3, nz=5, nb=8, src=(2, 1, 2)),
}


@pytest.fixture(autouse=True)
def _tma():
    import paper_1603_03971_gb300 as rtm

    yield
    rtm.set_tuning(4, 0, 0)
    rtm.set_tuning(8, 0, 0)


def _use(r, zchunk, variant=2):
    import paper_1603_03971_gb300 as rtm

    rtm.set_tuning(r, zchunk, variant)


# variant 2: 16-row tiles (256 threads); variant 3: 8-row tiles (128 threads)
@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("r", [4, 8])
@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("zchunk", [0, 16, 5])
def test_tma_forward_parity(r, shape, zchunk, variant):
    case = Case(r=r, nt=40, **SHAPES[shape])
    if shape == "thin":
        case.rec_stride = 1
    _use(r, zchunk, variant)
    g = DeviceShot(case)
    data, last = g.forward(keep_last=True)
    ref = case.oracle_problem().forward(keep_last=True)
    assert rel_l2(data.cpu().numpy(), ref["data"]) <= TOL
    assert rel_l2(last[1].cpu().numpy(), ref["last"][1]) <= TOL


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("r,storage,ck", [(4, "ckpt", 16), (8, "all", 0)])
def test_tma_backward_image_parity(r, storage, ck, variant):
    case = Case(r=r, nt=50, storage=storage, ckpt_every=ck, **SHAPES["ragged"])
    _use(r, 0, variant)
    g = DeviceShot(case)
    g.forward()
    d_obs = case.d_obs(g.nrec)
    img, adj = g.backward_image(d_obs, src_adj=True)
    prob = case.oracle_problem()
    fw = prob.forward(keep_u=True)
    bw = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=fw["u"])
    assert rel_l2(img.cpu().numpy(), bw["image"]) <= TOL
    assert rel_l2(adj.cpu().numpy(), bw["src_adj"]) <= TOL


@pytest.mark.parametrize("variant", [2, 3])
def test_tma_gradient_parity(variant):
    case = Case(r=4, nt=40, storage="ckpt", ckpt_every=9, **SHAPES["small"])
    _use(4, 0, variant)
    g = DeviceShot(case, want_grad=True, squared=True)
    g.forward()
    resid = case.d_obs(g.nrec)
    grad = g.grad(resid).cpu().numpy()
    prob = case.oracle_problem(squared=True)
    d_oracle = prob.forward()["data"]
    _, grad_ref = prob.misfit_and_grad(d_oracle - resid)
    assert rel_l2(grad, grad_ref) <= TOL


def test_tma_agrees_with_vector_loads():
    import paper_1603_03971_gb300 as rtm

    case = Case(r=4, nt=30, **SHAPES["ragged"])
    out = []
    for variant in (1, 2, 3):
        rtm.set_tuning(4, 0, variant)
        g = DeviceShot(case)
        data, last = g.forward(keep_last=True)
        out.append(last.cpu().numpy())
    assert rel_l2(out[1], out[0]) <= 1e-6
    # the tile shape changes no arithmetic
    assert np.array_equal(out[2], out[1])
