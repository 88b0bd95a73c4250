"""ctypes declarations of the C ABI in include/pargeo_gpu.h.

The shared library is built in-tree by `paper_2207_01834_gb300.build`.  There
is no fallback: if the library is missing or a call fails, an exception is
raised.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from .build import LIB

PG_OK, PG_EINVAL, PG_ENOMEM, PG_ECUDA, PG_ETIMEOUT, PG_EUNSUPPORTED = range(6)
STATUS_NAMES = {0: "PG_OK", 1: "PG_EINVAL", 2: "PG_ENOMEM", 3: "PG_ECUDA", 4: "PG_ETIMEOUT",
                5: "PG_EUNSUPPORTED"}
KNN_AUTO, KNN_THREAD, KNN_PACKET, KNN_POSTPONED, KNN_WARP, KNN_POSTPONED_HEAP = 0, 1, 2, 3, 4, 5
KNN_VARIANTS = (KNN_THREAD, KNN_PACKET, KNN_POSTPONED, KNN_WARP, KNN_POSTPONED_HEAP)
MAX_DIM = 16
MAX_K = 64
MAX_LEAF = 256
DEPTH_CAP = 48


class PgError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class TreeInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("dim", C.c_int32), ("dim_class", C.c_int32), ("leaf_size", C.c_int32),
                ("num_nodes", C.c_int32), ("depth", C.c_int32), ("node_floats", C.c_int32),
                ("point_floats", C.c_int32), ("root_ref", C.c_int32), ("root_cnt", C.c_int32),
                ("root_lo", C.c_float * MAX_DIM), ("root_hi", C.c_float * MAX_DIM)]


_P = C.c_void_p
_I64 = C.c_int64
_I = C.c_int
_S = C.c_int  # pg_status

SIGNATURES = {
    "pg_tree_build": (_S, [_P, _I64, _I, _I, _P, C.POINTER(_P)]),
    "pg_tree_build_split": (_S, [_P, _I64, _I, _I, _I, _P, C.POINTER(_P)]),
    "pg_knn": (_S, [_P, _P, _I64, _I, _P, _P, _P]),
    "pg_knn_ex": (_S, [_P, _P, _I64, _I, _I, _P, _P, _P]),
    "pg_knn_tune_set": (_S, [_I, _I, _I, _I]),
    "pg_knn_tune_get": (_S, [_I, _I, _I, C.POINTER(_I)]),
    "pg_tree_free": (_S, [_P]),
    "pg_tree_info": (_S, [_P, C.POINTER(TreeInfo)]),
    "pg_tree_export": (_S, [_P, _P, _P, _P, _P]),
    "pg_knn_set_variant": (_S, [_I]),
    "pg_knn_graph": (_S, [_P, _I, _I64, _P, C.POINTER(_I64), _P]),
    "pg_range": (_S, [_P, _P, _I64, C.c_float, _I64, _P, _P, C.POINTER(_I64), _P]),
    "pg_range_fill": (_S, [_P, _P, _I64, C.c_float, _P, _I64, _P, _P]),
    "pg_knn_touch_enable": (_S, [_I]),
    "pg_knn_touch_read": (_S, [C.POINTER(_I64), C.POINTER(_I64)]),
    "pg_bdl_create": (_S, [_I, _I64, _I, _P, C.POINTER(_P)]),
    "pg_bdl_insert": (_S, [_P, _P, _I64, _P]),
    "pg_bdl_erase": (_S, [_P, _P, _I64]),
    "pg_bdl_knn": (_S, [_P, _P, _I64, _I, _P, _P]),
    "pg_bdl_knn_ex": (_S, [_P, _P, _I64, _I, _I, _P, _P]),
    "pg_bdl_size": (_S, [_P, C.POINTER(_I64)]),
    "pg_bdl_structure": (_S, [_P, C.POINTER(C.c_uint64), _P, C.POINTER(_I64), C.POINTER(_I64)]),
    "pg_bdl_slot_of": (_S, [_P, _P]),
    "pg_bdl_free": (_S, [_P]),
    "pg_knn_backward": (_S, [_P, _I64, _P, _I64, _I, _I, _P, _P, _P, _P, _P]),
    "pg_knn_backward_noalloc": (_S, [_P, _I64, _P, _I64, _I, _I, _P, _P, _P, _P, _P]),
    "pg_batched_chamfer": (_S, [_P, _P, _P, _P, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P]),
    "pg_batched_chamfer_backward": (_S, [_P, _P, _P, _P, _I, _I, _I, _P, _P, _P, _P, _P, _P]),
    "pg_last_error": (C.c_char_p, []),
    "pg_version": (C.c_char_p, []),
    "pg_launch_count": (C.c_uint64, []),
    "pg_profile_enable": (_S, [_I]),
    "pg_profile_read": (_S, [C.c_char_p, C.POINTER(C.c_double), C.POINTER(_I64)]),
    "pg_debug_fail_alloc_after": (_S, [_I]),
    "pg_debug_batched_faults": (_S, [_I, C.c_longlong]),
}

_lock = threading.Lock()
_lib = None


def load():
    """Load libpargeo_gpu.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"{LIB} is missing: build the CUDA library first "
                                   "(python -m paper_2207_01834_gb300.build)")
            lib = C.CDLL(LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def call(name: str, *args) -> None:
    lib = load()
    st = getattr(lib, name)(*args)
    if st != PG_OK:
        msg = lib.pg_last_error().decode(errors="replace")
        raise PgError(st, name, msg)
