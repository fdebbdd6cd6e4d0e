"""ctypes declarations of the C ABI in include/hsearch.h (marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

HS_OK, HS_EINVAL, HS_ENOMEM, HS_ECUDA, HS_ETOOLONG, HS_ETIMEOUT, HS_ETRUNC, HS_EINTERNAL = range(8)
HS_MODE_DB = 0
HS_OP_M, HS_OP_I, HS_OP_D = 0, 1, 2
HS_MAX_QUERY_LEN = 2048
HS_MAX_K = 4096
HS_NOALLOC_SCRATCH_BYTES = 8 << 20

HIT_DTYPE = np.dtype([("db_index", "<i8"), ("score", "<i4"), ("q_begin", "<i4"), ("q_end", "<i4"),
                      ("t_begin", "<i4"), ("t_end", "<i4"), ("ops_len", "<i4"), ("ops_offset", "<i8")])
assert HIT_DTYPE.itemsize == 40


class hs_params(C.Structure):
    _fields_ = [("pgp", C.c_int32), ("gop", C.c_int32), ("gep", C.c_int32), ("rounds", C.c_int32),
                ("lfactor_q16", C.c_uint32), ("sfactor_q16", C.c_uint32), ("minfactor_q16", C.c_uint32),
                ("mode", C.c_int32), ("matrix", C.POINTER(C.c_int8))]


class hs_trace(C.Structure):
    _fields_ = [("scan_start", C.c_void_p), ("scan_stop", C.c_void_p), ("launches", C.c_int32),
                ("pack_shifts", C.c_int32)]


class hs_batch_tuning(C.Structure):
    _fields_ = [("chunks", C.c_int32), ("warps", C.c_int32), ("flat_min_chunks", C.c_int32),
                ("flat_max_iters", C.c_int32), ("long_len", C.c_int32)]


class HsError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = _L.hs_strerror(status).decode() if _L is not None else str(status)
        super().__init__("%s: %s (status %d)" % (where, msg, status))


_L = None


def lib():
    """The compiled library.  There is no fallback: if libhsearch.so is
    missing the call fails (build it with ``__graft_entry__.build()``)."""
    global _L
    if _L is not None:
        return _L
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libhsearch.so is not built (%s); run __graft_entry__.build()" % _build.LIB)
    L = C.CDLL(_build.LIB)
    P = C.POINTER
    vp, i32, i64, u64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_size_t
    L.hs_params_default.argtypes = [P(hs_params)]
    L.hs_params_default.restype = None
    L.hs_encode.argtypes = [C.c_char_p, i64, vp]
    L.hs_builtin_matrix.argtypes = [vp]
    L.hs_params_check.argtypes = [P(hs_params)]
    L.hs_db_load.argtypes = [vp, vp, i64, vp, P(vp)]
    L.hs_db_info.argtypes = [vp, P(i64), P(i64), P(i32)]
    L.hs_db_load_shard.argtypes = [vp, vp, i64, i64, vp, P(vp)]
    L.hs_db_index_base.argtypes = [vp, P(i64)]
    L.hs_db_set_schedule.argtypes = [vp, i32, vp]
    L.hs_db_get_schedule.argtypes = [vp, vp, vp]
    L.hs_search_threshold.argtypes = [vp, vp, i32, P(hs_params), i32, i32, u64, vp, vp, P(i32), P(i64), vp, i64, P(i64)]
    L.hs_db_free.argtypes = [vp]
    L.hs_db_free.restype = None
    L.hs_search_workspace_size.argtypes = [vp, i32, i32, P(sz)]
    L.hs_ops_capacity.argtypes = [i32, i32]
    L.hs_ops_capacity.restype = i64
    L.hs_search_device.argtypes = [vp, vp, i32, P(hs_params), i32, u64, vp, vp, sz, vp, vp, i64, vp, vp, vp, vp]
    L.hs_search.argtypes = [vp, vp, i32, P(hs_params), i32, u64, vp, vp, P(i32), vp, i64, P(i64)]
    L.hs_get_alignment.argtypes = [vp, vp, i32, P(hs_params), u64, i64, vp, vp, i64, P(i32), P(i64), vp]
    L.hs_search_device_noalloc.argtypes = [vp, vp, i32, P(hs_params), i32, u64, vp, vp, vp, i64, vp, vp, vp, vp]
    L.hs_search_transfer_bytes.argtypes = [i32, i32, P(i64), P(i64)]
    L.hs_search_batch_workspace_size.argtypes = [vp, i32, i64, i32, i32, P(sz)]
    L.hs_batch_ops_capacity.argtypes = [i32, i64, i32]
    L.hs_batch_ops_capacity.restype = i64
    L.hs_search_batch_device.argtypes = [vp, i32, vp, vp, vp, i64, i32, P(hs_params), i32, P(hs_batch_tuning), vp,
                                         vp, sz, vp, vp, i64, vp, vp]
    L.hs_search_batch.argtypes = [vp, i32, vp, vp, vp, P(hs_params), i32, P(hs_batch_tuning), vp, vp, P(i32), vp,
                                  i64, P(i64)]
    L.hs_db_set_trace.argtypes = [vp, P(hs_trace)]
    L.hs_strerror.argtypes = [C.c_int]
    L.hs_strerror.restype = C.c_char_p
    for name in ("hs_encode", "hs_builtin_matrix", "hs_params_check", "hs_db_load", "hs_db_info",
                 "hs_search_workspace_size", "hs_search_device", "hs_search", "hs_get_alignment",
                 "hs_search_transfer_bytes", "hs_db_set_trace", "hs_search_device_noalloc",
                 "hs_db_load_shard", "hs_db_index_base", "hs_search_threshold",
                 "hs_search_batch_workspace_size", "hs_search_batch_device", "hs_search_batch",
                 "hs_db_set_schedule", "hs_db_get_schedule"):
        getattr(L, name).restype = C.c_int
    _L = L
    return L


def check(status, where):
    if status != HS_OK:
        raise HsError(status, where)
