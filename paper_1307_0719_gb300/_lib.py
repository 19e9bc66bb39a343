"""ctypes binding of libtaylens.so (include/taylens.h): argument marshalling only."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libtaylens.so")

# status codes
TL_OK, TL_ERR_ARG, TL_ERR_NOMEM, TL_ERR_CUDA, TL_ERR_TIMEOUT, TL_ERR_UNSUPPORTED = range(6)
TL_SPIN_T, TL_SPIN_QU = 1, 2
TL_FP64, TL_MIXED_FP32, TL_MIXED_TF32, TL_MIXED_TF32x3, TL_MIXED_BF16x3 = range(5)
TL_ROTATE, TL_NAIVE, TL_EXPAND_AT_PIXEL = 1, 2, 4
TL_BATCH_LOOP, TL_BATCH_PERSISTENT, TL_BATCH_GRAPH = 0, 1, 2

# every symbol include/taylens.h declares, with its ctypes signature
_P = ctypes.c_void_p
SIGNATURES = {
    "tl_plan_create": (ctypes.c_int, [ctypes.c_int] * 6 + [ctypes.POINTER(ctypes.c_void_p)]),
    "tl_plan_destroy": (ctypes.c_int, [_P]),
    "tl_plan_workspace_bytes": (ctypes.c_size_t, [_P]),
    "tl_plan_maps_per_field": (ctypes.c_int, [_P]),
    "tl_plan_batch": (ctypes.c_int, [_P]),
    "tl_plan_batch_launches": (ctypes.c_longlong, [_P, ctypes.c_int, ctypes.c_int]),
    "tl_plan_device_error": (ctypes.c_int, [_P]),
    "tl_plan_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "tl_plan_set_lmax_phi": (ctypes.c_int, [_P, ctypes.c_int]),
    "tl_synth_derivs": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
    "tl_deflection": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "tl_lens": (ctypes.c_int, [_P] * 9),
    "tl_lens_host": (ctypes.c_int, [_P] * 9),
    "tl_lens_batch": (ctypes.c_int, [_P, ctypes.c_int] + [_P] * 8),
    "tl_lens_batch_host": (ctypes.c_int, [_P, ctypes.c_int] + [_P] * 8),
    "tl_lens_adjoint": (ctypes.c_int, [_P] * 14),
    "tl_deflection_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
    "tl_map2alm": (ctypes.c_int, [_P] * 8),
    "tl_anafast": (ctypes.c_int, [ctypes.c_int] + [_P] * 5),
    "tl_batch_create": (ctypes.c_int, [ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "tl_batch_destroy": (ctypes.c_int, [_P]),
    "tl_batch_lens": (ctypes.c_int, [_P, ctypes.c_int] + [_P] * 8),
    "tl_batch_autotune": (ctypes.c_int, [_P] * 9),
    "tl_batch_groups": (ctypes.c_int, [_P]),
    "tl_batch_waves": (ctypes.c_int, [_P]),
    "tl_batch_grid": (ctypes.c_int, [_P]),
    "tl_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tl_last_stage_ms": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
}

_lib = None


class TaylensError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {lib().tl_status_string(status).decode()} (status {status})")


def lib():
    """Load the in-tree library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                              "(python -m paper_1307_0719_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, what: str):
    if status != TL_OK:
        raise TaylensError(status, what)
