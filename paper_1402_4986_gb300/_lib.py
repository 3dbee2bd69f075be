"""ctypes declarations of the C ABI in ``include/idw.h``.

Loading fails loudly when the compiled library is missing: there is no CPU
fallback.  Build it with ``python -m paper_1402_4986_gb300.build`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_void_p = ctypes.c_void_p
c_int = ctypes.c_int
c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_double = ctypes.c_double
c_size_t = ctypes.c_size_t

STATUS = {
    0: "IDW_OK",
    1: "IDW_ERR_INVALID_ARG",
    2: "IDW_ERR_ALIGNMENT",
    3: "IDW_ERR_CUDA",
    4: "IDW_ERR_NOT_FINITE_INPUT",
    5: "IDW_ERR_WORKSPACE",
    6: "IDW_ERR_UNSUPPORTED",
    7: "IDW_ERR_DEVICE_TIMEOUT",
}
PREC_F32_COMP = 0
PREC_F64_PLAIN = 1
PAPER_KERNELS = {"naive": 0, "tiled": 1}
PAPER_LAYOUTS = {"soa": 0, "aos": 1, "aoas": 2, "hybrid": 3}
OPTIONS = {"autotune": 1, "sweep_variant": 2, "force_general_power": 3, "last_variant": 4,
           "tuned_classes": 5, "staging_layout": 6, "validate_inputs": 7,
           "local_query_order": 8, "deterministic": 9, "fma_log2": 10, "knn_search": 11}


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("queries_per_thread", c_int32),
        ("threads_per_cta", c_int32),
        ("queries_per_cta", c_int32),
        ("records_per_tile", c_int32),
        ("query_tiles", c_int64),
        ("data_tiles", c_int64),
        ("units", c_int64),
        ("grid", c_int32),
        ("max_pieces_per_query_tile", c_int32),
        ("partial_slots", c_int64),
        ("workspace_bytes", c_size_t),
    ]


# name -> (restype, argtypes); every symbol include/idw.h declares.
SIGNATURES = {
    "idw_status_string": (ctypes.c_char_p, [c_int]),
    "idw_create": (c_int, [ctypes.POINTER(c_void_p), c_int]),
    "idw_destroy": (c_int, [c_void_p]),
    "idw_last_cuda_error": (ctypes.c_char_p, [c_void_p]),
    "idw_interpolate": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_double, c_int,
                                c_void_p, c_void_p]),
    "idw_interpolate_saved": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_double,
                                      c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "idw_interpolate_host": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_double,
                                     c_int, c_void_p, c_void_p]),
    "idw_interpolate_batched": (c_int, [c_void_p, c_int32, ctypes.POINTER(c_void_p),
                                        ctypes.POINTER(c_int64), ctypes.POINTER(c_void_p),
                                        ctypes.POINTER(c_int64), c_double, c_int,
                                        ctypes.POINTER(c_void_p), c_void_p]),
    "idw_backward": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_double, c_void_p,
                             c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                             c_void_p, c_void_p]),
    "idw_sync_status": (c_int, [c_void_p, c_void_p]),
    "idw_plan_forward": (c_int, [c_int32, c_int32, c_int64, c_int64, c_double, c_int,
                                 ctypes.POINTER(PlanInfo)]),
    "idw_measure_pipe_rates": (c_int, [c_int, ctypes.POINTER(c_double)]),
    "idw_measure_mufu_errors": (c_int, [c_int, ctypes.POINTER(c_double)]),
    "idw_debug_check_failures": (c_int, [c_int, ctypes.POINTER(ctypes.c_uint32)]),
    "idw_set_option": (c_int, [c_void_p, c_int, c_int64]),
    "idw_get_option": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int64)]),
    "idw_profile_enable": (c_int, [c_void_p, c_int]),
    "idw_profile_read": (c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int64)]),
    "idw_selftest_bounded_wait": (c_int, [c_void_p, c_void_p]),
    "idw_paper_interpolate": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int64, c_void_p, c_int64,
                                      c_double, c_int, c_void_p, c_void_p]),
    "idw_interpolate_noalloc": (c_int, [c_void_p, c_int64, c_void_p, c_int64, c_double, c_void_p,
                                        c_void_p]),
    "idw_noalloc_sync_status": (c_int, [c_void_p]),
    "idw_noalloc_selftest_bounded_wait": (c_int, [c_void_p]),
    "idw_interpolate_local": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_double,
                                      c_double, c_void_p, c_void_p, c_void_p]),
    "idw_create_ex": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.c_char_p]),
    "idw_interpolate_knn": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_double,
                                    c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "idw_local_index_create": (c_int, [c_void_p, c_void_p, c_int64, c_double, c_int32,
                                       ctypes.POINTER(c_void_p), c_void_p]),
    "idw_local_index_interpolate": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_double,
                                            c_double, c_void_p, c_void_p, c_void_p]),
    "idw_local_index_modified": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_double,
                                         c_double, c_void_p, c_void_p, c_void_p]),
    "idw_local_index_knn": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_double, c_int32,
                                    c_void_p, c_void_p, c_void_p, c_void_p]),
    "idw_local_index_destroy": (c_int, [c_void_p]),
    "idw_local_backward": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_double,
                                   c_double, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p]),
    "idw_interpolate_modified": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64,
                                         c_double, c_double, c_void_p, c_void_p, c_void_p]),
    "idw_modified_backward": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_double,
                                      c_double, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p]),
    "idw_knn_backward": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_double,
                                 c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 c_void_p]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    """The library to load: the debug build (index checks, see
    idw_debug_check_failures) when IDW_DEBUG_CHECKS=1, else the release one."""
    return _build.LIB_DEBUG if os.environ.get("IDW_DEBUG_CHECKS") == "1" else _build.LIB


def load():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise ImportError(
                    f"the IDW CUDA library is not built ({path} is missing); run "
                    "`python -m paper_1402_4986_gb300.build` first. There is no CPU fallback.")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class IDWError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        self.name = STATUS.get(status, f"status {status}")
        super().__init__(f"{where}: {self.name}{(' (' + detail + ')') if detail else ''}")


def check(status: int, where: str, handle=None):
    if status != 0:
        detail = ""
        if status == 3 and handle is not None:
            detail = load().idw_last_cuda_error(handle).decode()
        raise IDWError(status, where, detail)
