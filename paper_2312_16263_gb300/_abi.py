"""ctypes binding of include/fwh.h (argument marshalling only).

Every function here has the name and the arguments of the C entry point it
wraps; all computation happens in the CUDA library.  Loading fails loudly if
the library has not been built (there is no fallback implementation).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libfwh_gb300.so")

FWH_OK, FWH_ERR_ARG, FWH_ERR_CUDA, FWH_ERR_OOM, FWH_ERR_STATE, FWH_ERR_TIMEOUT = range(6)
FWH_FP64, FWH_MIXED = 0, 1
FWH_BATCH_PIPELINED, FWH_BATCH_GRID, FWH_BATCH_PERSISTENT = 0, 1, 2
STATUS_NAMES = {0: "FWH_OK", 1: "FWH_ERR_ARG", 2: "FWH_ERR_CUDA", 3: "FWH_ERR_OOM",
                4: "FWH_ERR_STATE", 5: "FWH_ERR_TIMEOUT"}

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_ip64 = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); mirrors include/fwh.h
SIGNATURES = {
    "fwh_create": (ctypes.c_int, [ctypes.POINTER(_vp), _i64, _vp, _vp, _vp, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int]),
    "fwh_set_observers": (ctypes.c_int, [_vp, _i64, _vp]),
    "fwh_forward": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "fwh_forward_noalloc": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "fwh_observer_window": (ctypes.c_int, [_vp, _i64, _dp, _ip64]),
    "fwh_observer_extremes": (ctypes.c_int, [_vp, _dp, _dp]),
    "fwh_set_observer_extremes": (ctypes.c_int, [_vp, _dp, _dp]),
    "fwh_backward": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "fwh_batch_forward": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_vp),
                                         ctypes.POINTER(_vp), _ip64, ctypes.POINTER(_vp),
                                         _vp]),
    "fwh_autotune": (ctypes.c_int, [_vp, _i64, ctypes.POINTER(ctypes.c_int), _vp]),
    "fwh_set_tile_config": (ctypes.c_int, [_vp, ctypes.c_int]),
    "fwh_set_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "fwh_set_pipeline": (ctypes.c_int, [_vp, ctypes.c_int]),
    "fwh_set_batch_options": (ctypes.c_int, [_vp, _i64, ctypes.c_int]),
    "fwh_set_wait_limit": (ctypes.c_int, [_vp, _i64, ctypes.c_int]),
    "fwh_last_timings": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float)]),
    "fwh_timing_totals": (ctypes.c_int, [_vp, _dp, _ip64, ctypes.c_int]),
    "fwh_check": (ctypes.c_int, [_vp, _vp]),
    "fwh_fma_peak": (ctypes.c_int, [ctypes.c_int, _dp, _vp]),
    "fwh_forward_moving": (ctypes.c_int, [_i64, _i64, _vp, _vp, _vp, _vp, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, _vp, _i64, _vp,
                                          _vp, _vp, _dp, _ip64, _vp]),
    "fwh_set_moving_scratch": (ctypes.c_int, [_i64]),
    "fwh_psd": (ctypes.c_int, [_i64, _vp, _i64, _vp, ctypes.c_double, _i64, ctypes.c_int,
                               ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "fwh_get_sizes": (ctypes.c_int, [_vp, _ip64, _ip64, ctypes.POINTER(ctypes.c_int)]),
    "fwh_destroy": (None, [_vp]),
    "fwh_last_error": (ctypes.c_char_p, [_vp]),
    "fwh_version": (ctypes.c_char_p, []),
}

_lib = None


class FWHError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it is missing (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"FW-H CUDA library not found at {path}; build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, handle=None):
    if status != FWH_OK:
        msg = load().fwh_last_error(handle)
        raise FWHError(status, msg.decode() if msg else "")
    return status
