"""ctypes binding to libplv.so (the C ABI of include/plv.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind these entry points.  There is no CPU fallback: if the library
is missing or a call fails, a ``PlvError`` is raised.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PLV_OK = 0
PLV_ERR_INVALID = 1
PLV_ERR_ALLOC = 2
PLV_ERR_CUDA = 3
PLV_ERR_UNSUPPORTED = 4
PLV_ERR_TIMEOUT = 5
PLV_ERR_NUMERIC = 6

PLV_F32 = 0
PLV_F64 = 1
PLV_PREC_FP32 = 0
PLV_PREC_BF16X3 = 1
PLV_PREC_FP16X3 = 2
PLV_OUT_PLV = 1
PLV_OUT_IPLV = 2
PLV_OUT_CIPLV = 4
PLV_OUT_C = 8
PLV_TRIAL_ASIS = 0
PLV_TRIAL_RMS = 1
PLV_FAULT_NONE = 0
PLV_FAULT_ALLOC = 1
PLV_FAULT_LAUNCH = 2
PLV_FAULT_STALL = 3

STATUS_NAMES = {0: "PLV_OK", 1: "PLV_ERR_INVALID", 2: "PLV_ERR_ALLOC",
                3: "PLV_ERR_CUDA", 4: "PLV_ERR_UNSUPPORTED",
                5: "PLV_ERR_TIMEOUT", 6: "PLV_ERR_NUMERIC"}

# every entry point include/plv.h declares: name -> (restype, argtypes)
_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_u = ctypes.c_uint
_sz = ctypes.c_size_t
SIGNATURES = {
    "plv_create": (_i, [ctypes.POINTER(_vp), _i, _i, _sz]),
    "plv_destroy": (_i, [_vp]),
    "plv_last_error": (ctypes.c_char_p, [_vp]),
    "plv_get_precision": (_i, [_vp]),
    "plv_set_gram_raster": (_i, [_vp, _i]),
    "plv_set_wait_limit": (_i, [_vp, ctypes.c_uint64]),
    "plv_memory_usage": (_i, [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_sz)]),
    "plv_check_status": (_i, [_vp, _vp, ctypes.POINTER(_i)]),
    "plv_build_checked": (_i, []),
    "plv_debug_fault": (_i, [_i, _i]),
    "plv_debug_fault_armed": (_i, [ctypes.POINTER(_i)]),
    "plv_phasor_ld": (_i64, [_i]),
    "plv_phasor_bytes": (_sz, [_vp, _i, _i, _i]),
    "plv_prepare": (_i, [_vp, _i]),
    "plv_analytic": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i64, _vp]),
    "plv_normalize": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i64, _vp]),
    "plv_gram": (_i, [_vp, _vp, _vp, _i, _i, _i, _u, _vp, _vp, _vp, _vp,
                      _vp]),
    "plv_metrics": (_i, [_vp, _vp, _vp, _i, _i, _vp, _vp, _vp]),
    "plv_backward": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i64, _vp, _vp, _vp,
                          _vp, _vp]),
    "plv_backward_noalloc": (_i, [_vp, _vp, _i, _i, _i, _i, _i64, _vp, _vp,
                                  _vp, _vp, _vp]),
    "plv_group_create": (_i, [_vp, _vp, _i, _u, ctypes.POINTER(_vp)]),
    "plv_gram_grouped": (_i, [_vp, _vp, _vp]),
    "plv_analytic_grouped": (_i, [_vp, _vp, _vp]),
    "plv_trial_operands": (_i, [_vp, _vp, _vp, _i, _i, _i64, _i, _i, _i, _vp]),
    "plv_analytic_bands": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i64, _vp, _i, _vp]),
    "plv_dft_bins": (_i, [_vp, _vp, _vp, _i, _i, _i, _i64, _i, _i, _vp, _i64]),
    "plv_gram_windows": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _u, _vp, _vp, _vp,
                              _vp, _vp]),
    "plv_group_tune": (_i, [_vp, _vp, _vp, _i, _vp]),
    "plv_group_configure": (_i, [_vp, _vp, _vp, _i, _vp, _i, _i, _i]),
    "plv_gram_split_plan": (_i, [_vp, _i, _i, _i, _i, _vp]),
    "plv_analytic_save": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i64, _vp, _vp, _vp]),
    "plv_backward_saved": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "plv_group_destroy": (_i, [_vp]),
    "plv_sync_status": (_i, [_vp, _vp, ctypes.POINTER(_i)]),
}

_lock = threading.Lock()
_libs = {}


class PlvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib_path(checked: bool = False) -> str:
    return _build.LIB_CHECKED if checked else _build.LIB


def load(build_if_missing: bool = True, checked: bool = False):
    """Load (building first if needed) libplv.so -- or, with checked=True,
    the bounds-checked libplv_checked.so -- and declare signatures."""
    with _lock:
        if checked not in _libs:
            path = lib_path(checked)
            if build_if_missing and not _build.up_to_date(checked):
                _build.build(checked=checked)
            if not os.path.exists(path):
                raise PlvError(PLV_ERR_UNSUPPORTED,
                               f"CUDA library not built: {path}")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _libs[checked] = lib
    return _libs[checked]


# handles created by the checked library (their error text lives there)
_checked_handles = set()


def check(status: int, handle=None, lib=None):
    if status != PLV_OK:
        if lib is None:
            hv = getattr(handle, "value", handle)
            lib = load(checked=True) if hv in _checked_handles else load()
        msg = lib.plv_last_error(handle)
        raise PlvError(status, msg.decode() if msg else "")


class PlvTuneResult(ctypes.Structure):
    """Mirror of plv_tune_result (include/plv.h)."""
    _fields_ = [("k1_ms_default", ctypes.c_float),
                ("k1_ms_tuned", ctypes.c_float),
                ("gram_ms_default", ctypes.c_float),
                ("gram_ms_tuned", ctypes.c_float),
                ("k1_lengths", ctypes.c_int), ("k1_widened", ctypes.c_int),
                ("k1_per_sm", ctypes.c_int * 4),
                ("k1_launches", ctypes.c_int),
                ("gram_schedule", ctypes.c_int),
                ("gram_tile_cost", ctypes.c_int),
                ("gram_split", ctypes.c_int),
                ("gram_split_tiles", ctypes.c_int),
                ("timed_configs", ctypes.c_int), ("cached", ctypes.c_int)]


class PlvProblem(ctypes.Structure):
    """Mirror of plv_problem (include/plv.h)."""
    _fields_ = [("P", ctypes.c_void_p), ("batch", ctypes.c_int),
                ("N", ctypes.c_int), ("T", ctypes.c_int),
                ("plv", ctypes.c_void_p), ("iplv", ctypes.c_void_p),
                ("ciplv", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("diag", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("ldx", ctypes.c_int64), ("dtype", ctypes.c_int)]
