"""Post-run scan of the fields for non-finite values: a forward pass whose
coefficients hold a NaN, or whose coefficients are far past the stability
limit, ends with RTM_ERR_NUMERIC in the device status word (rtm_check); a
clean run does not. The NaN and the blow-up are ordinary floating-point
values: nothing here faults."""
import numpy as np
import pytest

from helpers import Case, DeviceShot

pytestmark = pytest.mark.gpu


def _status_after(g, c):
    import torch

    from paper_1603_03971_gb300 import _lib

    data = torch.empty((g.p.nt, g.nrec), dtype=torch.float32, device=g.dev)
    g.rtm.forward(g.p, c, g.rec, g.ws, data=data)
    try:
        g.rtm.check(g.ws)
        return 0
    except _lib.RtmError as e:
        return e.code


@pytest.mark.parametrize("r", [4, 8])
def test_clean_run_passes_the_scan(r):
    g = DeviceShot(Case(r=r, nt=30))
    assert _status_after(g, g.c) == 0


@pytest.mark.parametrize("r", [4, 8])
def test_nan_coefficient_is_reported(r):
    g = DeviceShot(Case(r=r, nt=30))
    c = g.c.clone()
    flat = c.view(-1)
    flat[flat.numel() // 2] = float("nan")
    assert _status_after(g, c) == 6  # RTM_ERR_NUMERIC
    # the status word was cleared by the check: a clean run passes again
    assert _status_after(g, g.c) == 0


def test_unstable_coefficients_are_reported():
    # c = v^2 dt^2 scaled far past the stability limit: the leapfrog grows by
    # orders of magnitude per step and overflows within the run
    g = DeviceShot(Case(r=4, nt=200))
    c = g.c * 400.0
    assert _status_after(g, c) == 6


def test_backward_scans_the_image():
    import torch

    case = Case(r=4, nt=30)
    g = DeviceShot(case)
    g.forward()
    d = np.full((case.nt, g.nrec), np.nan, dtype=np.float32)
    rd = torch.from_numpy(d).to(g.dev)
    img = torch.zeros((case.nz, case.ny, case.nx), dtype=torch.float32, device=g.dev)
    g.rtm.backward_image(g.p, g.c, g.rec, rd, g.ws, img)
    from paper_1603_03971_gb300 import _lib

    with pytest.raises(_lib.RtmError) as e:
        g.rtm.check(g.ws)
    assert e.value.code == 6
