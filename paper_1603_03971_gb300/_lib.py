"""ctypes binding of librtm (include/rtm.h): argument marshalling only.

Loading fails loudly if the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librtm.so")

RTM_OK = 0
STATUS_NAMES = {
    0: "RTM_OK", 1: "RTM_ERR_INVALID", 2: "RTM_ERR_CFL", 3: "RTM_ERR_WORKSPACE",
    4: "RTM_ERR_CUDA", 5: "RTM_ERR_TIMEOUT", 6: "RTM_ERR_NUMERIC", 7: "RTM_ERR_UNSUPPORTED",
    8: "RTM_ERR_STATE",
}
(RTM_STORE_ALL, RTM_STORE_CKPT, RTM_STORE_LEARNED, RTM_STORE_REVOLVE, RTM_STORE_BOUNDARY,
 RTM_STORE_DECIMATED) = 0, 1, 2, 3, 4, 5
RTM_VEL_V, RTM_VEL_V2 = 0, 1


class RtmParams(ctypes.Structure):
    """Mirror of ``rtm_params``."""

    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("nb", ctypes.c_int32), ("radius", ctypes.c_int32), ("nt", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("f0", ctypes.c_double),
        ("t0", ctypes.c_double),
        ("src_x", ctypes.c_int32), ("src_y", ctypes.c_int32), ("src_z", ctypes.c_int32),
        ("nrec", ctypes.c_int32), ("storage", ctypes.c_int32), ("ckpt_every", ctypes.c_int32),
        ("image_every", ctypes.c_int32), ("want_grad", ctypes.c_int32),
    ]

    def copy(self, **changes) -> "RtmParams":
        q = RtmParams()
        ctypes.pointer(q)[0] = self
        for k, v in changes.items():
            setattr(q, k, v)
        return q

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class RtmStats(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int64),
        ("stencil_launches", ctypes.c_int64 * 7),
        ("stencil_ms", ctypes.c_double * 7),
        ("stencil_bytes", ctypes.c_double * 7),
    ]


class RtmError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        self.code = code
        super().__init__("%s -> %s: %s" % (func, STATUS_NAMES.get(code, code), msg))


_lib = None

# symbol -> (restype, argtypes)
_P = ctypes.POINTER(RtmParams)
_vp, _sz, _i32, _i64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int64
SIGNATURES = {
    "rtm_version": (ctypes.c_char_p, []),
    "rtm_last_error": (ctypes.c_char_p, []),
    "rtm_validate": (ctypes.c_int, [_P]),
    "rtm_workspace_size": (_sz, [_P]),
    "rtm_model_prep": (ctypes.c_int, [_P, _vp, _i32, _vp, _vp, _sz, _vp]),
    "rtm_forward": (ctypes.c_int, [_P, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "rtm_backward_image": (ctypes.c_int, [_P, _vp, _vp, _vp, _vp, _sz, _vp, _vp, _vp]),
    "rtm_shot": (ctypes.c_int, [_P, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "rtm_grad": (ctypes.c_int, [_P, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "rtm_misfit": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "rtm_host_workspace_size": (_sz, [_P]),
    "rtm_shot_host": (ctypes.c_int, [_P, _vp, _i32, _vp, _vp, _vp, _vp, _sz, _vp]),
    "rtm_check": (ctypes.c_int, [_vp, _sz, _vp]),
    "rtm_forward_noalloc": (ctypes.c_int, [_P, _vp, _vp, _vp, _vp, _vp]),
    "rtm_set_tuning": (ctypes.c_int, [_i32, _i32, _i32]),
    "rtm_set_tuning_mode": (ctypes.c_int, [_i32, _i32, _i32]),
    "rtm_set_test_stall": (ctypes.c_int, [_i32, _i32]),
    "rtm_offgrid_taps": (_sz, [_P, _vp, _i32, _vp, _vp, _sz]),
    "rtm_forward_offgrid": (ctypes.c_int, [_P, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "rtm_shot_offgrid": (ctypes.c_int, [_P, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "rtm_decomp_plan": (ctypes.c_int32, [_P, _i32, _i32, _vp, _i32]),
    "rtm_decomp_workspace_size": (_sz, [_P, _i32, _i32]),
    "rtm_forward_decomposed": (ctypes.c_int, [_P, _i32, _i32, _vp, _vp, _vp, _vp, _sz, _vp,
                                              _vp]),
    "rtm_forward_learned": (ctypes.c_int, [_P, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "rtm_backward_image_learned": (ctypes.c_int, [_P, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "rtm_shot_learned": (ctypes.c_int, [_P, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "rtm_snapshot": (ctypes.c_int, [_P, _vp, _sz, _i32, _vp, _vp]),
    "rtm_batch_workspace_size": (_sz, [_P, _i32, _vp, _sz]),
    "rtm_batch_set_wait": (ctypes.c_int, [ctypes.c_double, _i32]),
    "rtm_batch": (ctypes.c_int, [_P, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _sz, _i32, _vp]),
    "rtm_backward_image_illum": (ctypes.c_int, [_P, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _vp,
                                                _vp]),
    "rtm_image_filter": (ctypes.c_int, [_P, _vp, _vp, ctypes.c_float, _vp, _vp, _vp, _sz, _vp]),
    "rtm_revolve_cost": (ctypes.c_int64, [_i32, _i32]),
    "rtm_revolve_schedule": (ctypes.c_int32, [_i32, _i32, _vp, _i32]),
    "rtm_ae_param_count": (_sz, []),
    "rtm_ae_workspace_size": (_sz, [_i32, _i32, _i32]),
    "rtm_ae_encode": (ctypes.c_int, [_vp, _vp, _i64, _i64, _i32, _i32, _i32, _vp, _vp, _vp, _sz,
                                     _vp]),
    "rtm_ae_decode": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _i64, _i32, _i32, _i32, _vp, _sz,
                                     _vp]),
    "rtm_ae_train_step": (ctypes.c_int, [_vp, _vp, _vp, _i32, ctypes.c_float, _vp, _i32, _i32,
                                         _i32, _i32, _vp, _vp, _vp, _sz, _vp]),
    "rtm_ae_gemm_bf16": (ctypes.c_int, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "rtm_ae_set_decoder": (ctypes.c_int, [_i32]),
    "rtm_ae_set_encoder": (ctypes.c_int, [_i32]),
    "rtm_set_timing": (ctypes.c_int, [_i32]),
    "rtm_stats_get": (ctypes.c_int, [ctypes.POINTER(RtmStats)]),
    "rtm_stats_reset": (ctypes.c_int, []),
}


def lib():
    """The loaded librtm; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "librtm is not built (%s missing): run `python -c \"import __graft_entry__ as g; "
                "g.build()\"` first" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def call(name: str, *args) -> int:
    """Call an entry point that returns rtm_status; raise RtmError unless OK."""
    rc = getattr(lib(), name)(*args)
    if rc != RTM_OK:
        msg = lib().rtm_last_error()
        raise RtmError(rc, name, msg.decode() if msg else "")
    return rc
