"""ctypes loader for libccl.so (the C ABI in include/ccl.h).

The library is built in-tree by ``paper_1708_08180_gb300.build``; importing a
function from here when it is missing raises instead of falling back to any
other implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

CCL_OK = 0
CCL_ERR_INVALID_ARG = 1
CCL_ERR_CUDA = 2
CCL_ERR_OOM = 3
CCL_ERR_TIMEOUT = 4
CCL_ERR_REJECTED = 5
CCL_ERR_SHUTDOWN = 6
CCL_ERR_NOT_FOUND = 7
CCL_ERR_PENDING = 8
CCL_FLAG_LOCAL_ONLY = 1
CCL_STATIC_SCRATCH_BYTES = 64 << 20
CCL_TILE_CLASSES = 7


class CclError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        name = status_string(status) if _lib is not None else str(status)
        super().__init__(f"{what}: {name}" if what else name)


class ccl_image(ctypes.Structure):
    _fields_ = [("d_img", ctypes.c_void_p), ("d_labels", ctypes.c_void_p),
                ("height", ctypes.c_int), ("width", ctypes.c_int)]


class ccl_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int),
                ("max_inflight", ctypes.c_int), ("connectivity", ctypes.c_int),
                ("device", ctypes.c_int)]


_c = ctypes
_P = _c.c_void_p
_SIGS = {
    "ccl_status_string": (_c.c_char_p, [_c.c_int]),
    "ccl_default_tile_width": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int]),
    "ccl_workspace_bytes": (_c.c_size_t, [_c.c_int, _c.c_int, _c.c_int]),
    "ccl_workspace_bytes_tiled": (_c.c_size_t, [_c.c_int, _c.c_int, _c.c_int, _c.c_int]),
    "ccl_label": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_int, _P, _c.c_size_t, _P]),
    "ccl_label_tiled": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_uint,
                                   _P, _c.c_size_t, _P]),
    "ccl_label_static": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_int, _P]),
    "ccl_label3d": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _P, _c.c_size_t,
                               _P]),
    "ccl_workspace_bytes3d": (_c.c_size_t, [_c.c_int, _c.c_int, _c.c_int, _c.c_int]),
    "ccl_label_regions": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_int, _P, _c.c_int, _P,
                                     _c.c_size_t, _P]),
    "ccl_stats_workspace_bytes": (_c.c_size_t, [_c.c_int, _c.c_int, _c.c_int]),
    "ccl_component_stats": (_c.c_int, [_P, _c.c_int, _c.c_int, _P, _c.c_int, _P, _P, _c.c_size_t,
                                       _P]),
    "ccl_label_with_stats": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_int, _P, _c.c_int, _P, _P,
                                        _c.c_size_t, _P]),
    "ccl_workspace_bytes_with_stats": (_c.c_size_t, [_c.c_int, _c.c_int, _c.c_int]),
    "ccl_seam_pair_count": (_c.c_longlong, [_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int]),
    "ccl_sync": (_c.c_int, [_P]),
    "ccl_get_tile_table": (_c.c_int, [_c.c_int, _c.POINTER(_c.c_int)]),
    "ccl_set_tile_table": (_c.c_int, [_c.c_int, _c.POINTER(_c.c_int)]),
    "ccl_autotune": (_c.c_int, [_c.c_int, _c.c_int, _P]),
    "ccl_set_phase_events": (None, [_c.POINTER(_P)]),
    "ccl_shutdown": (_c.c_int, []),
    "ccl_set_hop_budget": (_c.c_int, [_c.c_int, _c.c_int]),
    "ccl_inject_alloc_failures": (_c.c_int, [_c.c_int]),
    "ccl_batched_workspace_bytes": (_c.c_size_t, [_c.POINTER(ccl_image), _c.c_int, _c.c_int]),
    "ccl_label_batched": (_c.c_int, [_c.POINTER(ccl_image), _c.c_int, _c.c_int, _P, _c.c_size_t,
                                     _P]),
    "ccl_server_create": (_c.c_int, [_c.POINTER(ccl_server_config), _c.POINTER(_P)]),
    "ccl_server_submit": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _P, _c.POINTER(_c.c_uint64)]),
    "ccl_server_wait": (_c.c_int, [_P, _c.c_uint64, _c.c_int]),
    "ccl_server_poll": (_c.c_int, [_P, _c.c_uint64]),
    "ccl_server_stats": (_c.c_int, [_P, _c.POINTER(_c.c_double), _c.POINTER(_c.c_double),
                                    _c.POINTER(_c.c_double), _c.POINTER(_c.c_uint64),
                                    _c.POINTER(_c.c_uint64)]),
    "ccl_server_destroy": (_c.c_int, [_P]),
    "ccl_server_timing": (_c.c_int, [_P, _c.POINTER(_c.c_double), _c.POINTER(_c.c_double),
                                     _c.POINTER(_c.c_double), _c.POINTER(_c.c_uint64)]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libccl.so, building it first when allowed and missing/stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libccl.so not built ({path}); run "
                                   "python -m paper_1708_08180_gb300.build")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().ccl_status_string(int(status)).decode()


def check(status: int, what: str = "") -> None:
    if status != CCL_OK:
        raise CclError(status, what)
