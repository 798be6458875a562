"""rtm_forward_noalloc: forward modelling for callers that cannot allocate
device memory (a host application that owns every allocation, a plugin that
may not touch the process's allocator). Its scratch is a static device array
inside librtm; this file checks it against rtm_forward, which uses a caller
workspace, on two calls in a row (the array keeps the previous call's
contents, so the second call checks that the first is cleared away).

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import ctypes

import numpy as np
import pytest

from helpers import Case, DeviceShot, rel_l2

TOL = 1e-4


def _noalloc(p, c, rec, data, last):
    import torch

    from paper_1603_03971_gb300 import _lib

    _lib.call("rtm_forward_noalloc", ctypes.byref(p), ctypes.c_void_p(c.data_ptr()),
              ctypes.c_void_p(rec.data_ptr()), ctypes.c_void_p(data.data_ptr()),
              ctypes.c_void_p(last.data_ptr()),
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.gpu
def test_noalloc_forward_matches_workspace_forward_twice():
    import torch

    case = Case(r=4, nt=60, nx=100, ny=44, nz=37, nb=10)
    g = DeviceShot(case)
    data_ref, last_ref = g.forward(keep_last=True)
    for call in range(2):
        data = torch.full_like(data_ref, float("nan"))
        last = torch.full_like(last_ref, float("nan"))
        _noalloc(g.p, g.c, g.rec, data, last)
        torch.cuda.synchronize()
        assert rel_l2(data.cpu().numpy(), data_ref.cpu().numpy()) <= TOL, call
        assert rel_l2(last.cpu().numpy(), last_ref.cpu().numpy()) <= TOL, call
        assert np.isfinite(last.cpu().numpy()).all()


def test_noalloc_rejects_problems_larger_than_its_scratch():
    """The size check runs before any device work (no GPU needed)."""
    from paper_1603_03971_gb300 import _lib
    import paper_1603_03971_gb300 as rtm

    p = rtm.make_params(200, 200, 200, 20, 4, 10, 10.0, 1e-3, 20.0, 0.05, (100, 100, 4), 0)
    fake = ctypes.c_void_p(0x10000)  # never dereferenced
    rc = _lib.lib().rtm_forward_noalloc(ctypes.byref(p), fake, None, None, None, None)
    assert rc == 3
    assert b"static" in _lib.lib().rtm_last_error()
