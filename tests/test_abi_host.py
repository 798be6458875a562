"""Host-side checks of the C ABI: the library loads without a GPU, exports
every entry point that ``include/*.h`` declares, and rejects bad arguments
before touching the device."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

import paper_1603_03971_gb300 as rtm
from paper_1603_03971_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(rtm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rtm_forward", "rtm_backward_image", "rtm_shot", "rtm_grad",
                     "rtm_model_prep", "rtm_workspace_size", "rtm_misfit", "rtm_shot_host"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = _lib.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def _p(**kw):
    base = dict(nx=28, ny=24, nz=20, nb=6, radius=4, nt=40, dx=10.0, dt=1e-3, f0=20.0,
                t0=0.05, src=(3, 4, 5), nrec=10)
    base.update(kw)
    return rtm.make_params(**base)


def test_valid_params_pass():
    assert _lib.lib().rtm_validate(ctypes.byref(_p())) == 0


@pytest.mark.parametrize("change,code", [
    (dict(nx=0), 1), (dict(nb=-1), 1), (dict(radius=6), 7), (dict(nt=0), 1),
    (dict(dx=0.0), 1), (dict(dt=-1.0), 1), (dict(f0=0.0), 1),
    (dict(nx=27), 1),                      # nx + 2 nb not a multiple of 4
    (dict(src=(-7, 0, 0)), 1), (dict(src=(0, 30, 0)), 1), (dict(nrec=-1), 1),
    (dict(storage="ckpt", ckpt_every=0), 1), (dict(image_every=0), 1),
    (dict(want_grad=True, image_every=2), 1),
    (dict(storage="boundary", want_grad=True), 1),
    (dict(storage="boundary", nz=8), 1),  # model sides must exceed 2 r = 8
    (dict(storage="decimated", want_grad=True), 1),
    (dict(storage="decimated", ckpt_every=41), 1),  # exact window beyond nt
    (dict(storage="decimated", ckpt_every=-1), 1),
])
def test_invalid_params_rejected(change, code):
    p = _p(**change)
    assert _lib.lib().rtm_validate(ctypes.byref(p)) == code
    assert _lib.lib().rtm_workspace_size(ctypes.byref(p)) == 0
    assert len(_lib.lib().rtm_last_error()) > 0


def test_source_may_lie_in_the_sponge():
    assert _lib.lib().rtm_validate(ctypes.byref(_p(src=(-6, 29, 25)))) == 0


def test_calls_reject_bad_arguments_without_a_device():
    """Argument errors come back before any CUDA call (this runs without a GPU)."""
    L = _lib.lib()
    p = _p()
    n = L.rtm_workspace_size(ctypes.byref(p))
    fake = ctypes.c_void_p(0x10000)  # never dereferenced: validation fails first
    # workspace too small
    rc = L.rtm_forward(ctypes.byref(p), fake, fake, None, fake, n - 1, None, None)
    assert rc == 3
    # misaligned workspace
    rc = L.rtm_forward(ctypes.byref(p), fake, fake, None, ctypes.c_void_p(0x10010), n, None, None)
    assert rc == 3
    # NULL coefficients
    rc = L.rtm_forward(ctypes.byref(p), None, fake, None, fake, n, None, None)
    assert rc == 1
    # imaging call on a gradient workspace and vice versa
    pg = _p(want_grad=True)
    ng = L.rtm_workspace_size(ctypes.byref(pg))
    assert L.rtm_backward_image(ctypes.byref(pg), fake, fake, fake, fake, ng, fake, None, None) == 8
    assert L.rtm_grad(ctypes.byref(p), fake, fake, fake, fake, n, fake, None) == 8
    # misfit with negative length
    assert L.rtm_misfit(fake, fake, -1, None, fake, None) == 1
    assert L.rtm_set_tuning(6, 0, 0) == 7
    assert L.rtm_set_tuning(4, -1, 0) == 1
    assert L.rtm_set_tuning(4, 0, 4) == 1  # variants 0..3
    assert L.rtm_ae_set_decoder(3) == 1
    assert L.rtm_ae_set_decoder(-1) == 1
    assert L.rtm_ae_set_decoder(0) == 0
    assert L.rtm_ae_set_encoder(3) == 1
    assert L.rtm_ae_set_encoder(0) == 0
    # imaging variants: illumination output required; filter argument checks
    assert L.rtm_backward_image_illum(ctypes.byref(p), fake, fake, fake, None, fake, n, fake,
                                      None, None) == 1
    assert L.rtm_image_filter(ctypes.byref(p), None, fake, ctypes.c_float(1e-3), fake, None,
                              fake, 256, None) == 1
    assert L.rtm_image_filter(ctypes.byref(p), fake, None, ctypes.c_float(1e-3), fake, None,
                              fake, 256, None) == 1
    assert L.rtm_image_filter(ctypes.byref(p), fake, fake, ctypes.c_float(0.0), fake, None,
                              fake, 256, None) == 1
    assert L.rtm_image_filter(ctypes.byref(p), fake, fake, ctypes.c_float(1e-3), fake, None,
                              fake, 8, None) == 3
    p6 = _p()
    p6.radius = 6
    assert L.rtm_image_filter(ctypes.byref(p6), fake, None, ctypes.c_float(1e-3), None, fake,
                              None, 0, None) == 7


def test_workspace_sizes_follow_the_storage_policy():
    nx, ny, nz, nb, nt = 28, 24, 20, 6, 40
    N = (nx + 2 * nb) * (ny + 2 * nb) * (nz + 2 * nb)
    slab = nz * ny * (nx + 2 * nb)
    all_ = rtm.workspace_size(_p(nt=nt))
    # store-all keeps nt imaging snapshots of the model slab
    assert all_ >= 4 * (4 * N + slab + nt * slab)
    ck = rtm.workspace_size(_p(nt=nt, storage="ckpt", ckpt_every=16))
    # ceil(40/16) = 3 segments: 2 stored checkpoints of 2 fields, 16 snapshot slots
    assert ck >= 4 * (4 * N + slab + 2 * 2 * N + 16 * slab)
    assert ck < 4 * (4 * N + slab + 2 * 2 * N + 16 * slab) + 64 * 256
    # every-4th imaging keeps a quarter of the snapshots
    q = rtm.workspace_size(_p(nt=nt, image_every=4))
    assert q < all_ and q >= 4 * (4 * N + slab + (nt // 4) * slab)
    # the gradient keeps L u on the padded grid
    g = rtm.workspace_size(_p(nt=nt, want_grad=True))
    assert g >= 4 * (5 * N + nt * N)
    assert rtm.host_workspace_size(_p()) > all_
    # boundary storage: the band of u^1 .. u^{nt-2} and no snapshot slab
    r = 4
    band = 2 * r * nx * ny + 2 * r * (nz - 2 * r) * nx + 2 * r * (nz - 2 * r) * (ny - 2 * r)
    assert band == nx * ny * nz - (nx - 2 * r) * (ny - 2 * r) * (nz - 2 * r)
    b = rtm.workspace_size(_p(nt=nt, storage="boundary"))
    assert 4 * (4 * N + slab + (nt - 2) * band) <= b < 4 * (4 * N + slab + (nt - 2) * band) + 64 * 256


def test_test_stall_arms_and_disarms_without_a_device():
    """rtm_set_test_stall is host state only: it accepts the two kernels,
    arming (plane >= 0) and disarming (-1), and rejects an unknown kernel."""
    for kernel in (rtm.STALL_STENCIL, rtm.STALL_ENCODER):
        rtm.set_test_stall(kernel, 0)
        rtm.set_test_stall(kernel, -1)
    with pytest.raises(_lib.RtmError) as e:
        rtm.set_test_stall(7, 0)
    assert e.value.code == 1  # RTM_ERR_INVALID
