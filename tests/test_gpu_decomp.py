"""Forward modelling on an X-Y domain decomposition (subdomains with r-wide
halos, band launches first, halo pack / exchange / unpack on a communication
stream beside the interior launches) against the single-domain forward pass
(bit for bit: every cell sees the same arithmetic) and against the FP64
oracle (the wavefield tolerance)."""
import numpy as np
import pytest

from helpers import Case, DeviceShot, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(autouse=True)
def _reset_tuning():
    import paper_1603_03971_gb300 as rtm

    yield
    rtm.set_tuning(4, 0, 0)
    rtm.set_tuning(8, 0, 0)


def _decomposed(g, px, py):
    import torch

    import paper_1603_03971_gb300 as rtm

    ws = torch.empty(rtm.decomp_workspace_size(g.p, px, py), dtype=torch.uint8, device="cuda")
    data = torch.full((g.p.nt, g.nrec), float("nan"), device="cuda")
    last = torch.full((2,) + rtm.padded_shape(g.p), float("nan"), device="cuda")
    rtm.forward_decomposed(g.p, px, py, g.c, g.rec, ws, data=data, u_last=last)
    rtm.check(ws)
    return data, last


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("r", [4, 8])
@pytest.mark.parametrize("px,py", [(2, 1), (1, 2), (2, 2), (3, 2)])
def test_decomposed_forward_equals_the_single_domain_pass(variant, r, px, py):
    import paper_1603_03971_gb300 as rtm

    # 300 x 92 x 37 padded at nb = 10: several 64-wide band and interior
    # tiles per subdomain, ragged tails, and the source near a partition face
    case = Case(nx=280, ny=72, nz=17, nb=10, r=r, nt=40, src=(139, 35, 3), rec_stride=3)
    rtm.set_tuning(r, 0, variant)
    g = DeviceShot(case)
    data_ref, last_ref = g.forward(keep_last=True)
    data, last = _decomposed(g, px, py)
    assert np.array_equal(data.cpu().numpy(), data_ref.cpu().numpy())
    assert np.array_equal(last.cpu().numpy(), last_ref.cpu().numpy())


@pytest.mark.parametrize("r", [4, 8])
def test_decomposed_forward_matches_the_oracle(r):
    case = Case(nx=100, ny=44, nz=37, nb=10, r=r, nt=50, rec_stride=1)
    g = DeviceShot(case)
    data, last = _decomposed(g, 2, 2)
    ref = case.oracle_problem().forward(keep_last=True)
    assert rel_l2(data.cpu().numpy(), ref["data"]) <= TOL
    assert rel_l2(last[1].cpu().numpy(), ref["last"][1]) <= TOL
    assert rel_l2(last[0].cpu().numpy(), ref["last"][0]) <= TOL


def test_small_subdomains_are_all_band():
    """Subdomains narrower than two bands have no interior launch; 5 x 3
    subdomains of 24-cell columns and 15-row strips."""
    import paper_1603_03971_gb300 as rtm

    case = Case(nx=100, ny=24, nz=20, nb=10, r=4, nt=30)
    rtm.set_tuning(4, 0, 3)
    g = DeviceShot(case)
    data_ref, last_ref = g.forward(keep_last=True)
    data, last = _decomposed(g, 5, 3)
    assert np.array_equal(data.cpu().numpy(), data_ref.cpu().numpy())
    assert np.array_equal(last.cpu().numpy(), last_ref.cpu().numpy())


def test_receiver_outside_the_grid_is_reported():
    import paper_1603_03971_gb300 as rtm
    from paper_1603_03971_gb300 import _lib

    case = Case(r=4, nt=20, extra_rec=np.array([[500, 1, 2]], np.int32))
    g = DeviceShot(case)
    import torch

    ws = torch.empty(rtm.decomp_workspace_size(g.p, 2, 1), dtype=torch.uint8, device="cuda")
    data = torch.empty((g.p.nt, g.nrec), device="cuda")
    rtm.forward_decomposed(g.p, 2, 1, g.c, g.rec, ws, data=data)
    with pytest.raises(_lib.RtmError) as e:
        rtm.check(ws)
    assert e.value.code == 1
    assert float(data[:, -1].abs().max()) == 0.0
