"""Timeout paths of the kernels with mbarrier rings, on the GPU and without
a fault: rtm_set_test_stall makes one copy of the next launch expect 16
bytes more than it delivers, so the wait for that plane runs out after its
bound (about 2 s). The block raises its abort flag, waits (bounded) for
every copy it issued and leaves; the call's status word reads
RTM_ERR_TIMEOUT. Every copy lands, so nothing is left in flight: the device
stays usable and the next call, with the stall disarmed by the first
launch, is correct."""
import time

import numpy as np
import pytest

import rtm_inputs
from helpers import Case, DeviceShot

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("r", [4, 8])
def test_stencil_wait_timeout_is_reported_not_hung(r):
    import torch

    from paper_1603_03971_gb300 import _lib

    # checkpoint storage: the forward pass runs the plain forward step, the
    # kernel instance that takes the stall
    g = DeviceShot(Case(r=r, nt=6, storage="ckpt", ckpt_every=3))
    rtm = g.rtm
    rtm.set_tuning(r, 0, 3)  # the TMA stencil, 8-row tiles
    try:
        ref = torch.empty((g.p.nt, g.nrec), dtype=torch.float32, device=g.dev)
        rtm.forward(g.p, g.c, g.rec, g.ws, data=ref)
        rtm.check(g.ws)
        rtm.set_test_stall(rtm.STALL_STENCIL, 0)
        t0 = time.time()
        with pytest.raises(_lib.RtmError) as e:
            data = torch.empty_like(ref)
            rtm.forward(g.p, g.c, g.rec, g.ws, data=data)
            rtm.check(g.ws)
        assert e.value.code == 5  # RTM_ERR_TIMEOUT
        assert time.time() - t0 < 60
        # only one launch stalled; the next call clears the status and is exact
        again = torch.empty_like(ref)
        rtm.forward(g.p, g.c, g.rec, g.ws, data=again)
        rtm.check(g.ws)
        assert torch.equal(again, ref)
    finally:
        rtm.set_test_stall(rtm.STALL_STENCIL, -1)
        rtm.set_tuning(r, 0, 0)


def test_encoder_wait_timeout_is_reported_not_hung():
    import torch

    import paper_1603_03971_gb300 as rtm
    from paper_1603_03971_gb300 import _lib, codec

    shape = (64, 48, 40)
    P = torch.from_numpy(rtm_inputs.ae_flat(rtm_inputs.ae_init_params(3)).astype(np.float32))
    P = P.cuda()
    s = torch.from_numpy(rtm_inputs.standard_normal(shape, 71, np.float32)).cuda()
    codec.set_encoder("march")
    try:
        ws = codec.alloc_workspace(shape)
        l_ref, s_ref = codec.encode(P, s, ws)
        rtm.check(ws)
        rtm.set_test_stall(rtm.STALL_ENCODER, 0)
        t0 = time.time()
        ws_bad = codec.alloc_workspace(shape)
        with pytest.raises(_lib.RtmError) as e:
            codec.encode(P, s, ws_bad)
            rtm.check(ws_bad)
        assert e.value.code == 5  # RTM_ERR_TIMEOUT
        assert time.time() - t0 < 60
        # the codec's status word keeps an error until its workspace is new:
        # a fresh one shows the device usable and the next encode exact
        ws2 = codec.alloc_workspace(shape)
        l2, s2 = codec.encode(P, s, ws2)
        rtm.check(ws2)
        assert torch.equal(l2, l_ref) and torch.equal(s2, s_ref)
    finally:
        rtm.set_test_stall(rtm.STALL_ENCODER, -1)
        codec.set_encoder("auto")

