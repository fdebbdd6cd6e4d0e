"""GB300 heuristic protein database search (Nag & Karforma, arXiv 1508.06561).

Python binding of the C ABI in ``include/hsearch.h``.  It only marshals
arguments: every step of the search -- query profile, the pair-wise
heuristic alignment of Fig. 1 in database mode (Sec. III.B.3), ranking and
alignment replay -- runs in the library's CUDA kernels.  PyTorch supplies
device memory and streams for the device-resident entry point.

    db = Database(codes, offsets)               # load once (uint8 codes, int64 offsets)
    hits, ops = search(db, query, k=10)         # host in, host out
    out = search_device(db, q_cuda, k=10)       # torch tensors in HBM
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import _lib
from ._lib import HIT_DTYPE, HS_OP_D, HS_OP_I, HS_OP_M, HsError, check, lib

__all__ = ["Params", "Database", "search", "search_threshold", "search_batch", "search_batch_device",
           "search_device", "search_device_noalloc",
           "get_alignment", "encode",
           "builtin_matrix", "ops_to_rows", "HIT_DTYPE", "HsError", "workspace_size"]

GAP = 0xFF


@dataclass
class Params:
    """Sec. III.B.1 parameters; defaults are Sec. IV's (PGP=0, GOP=10, GEP=5,
    LFactor=0.5, SFactor=1, MinFactor=0.5) with Rounds=1 (Sec. III.B.3 a).
    Factors are Q16 fixed point (65536 == 1.0).  matrix: symmetric 24x24
    int8 (query letter, target letter); None = built-in BLOSUM62.  mode 1 is
    the pair-wise full-slide form of Fig. 1 (HS_MODE_FULL)."""
    pgp: int = 0
    gop: int = 10
    gep: int = 5
    rounds: int = 1
    lfactor_q16: int = 32768
    sfactor_q16: int = 65536
    minfactor_q16: int = 32768
    matrix: Optional[np.ndarray] = None
    mode: int = 0                       # 0: database search (Sec. III.B.3), 1: full slide (Fig. 1)

    def to_c(self):
        p = _lib.hs_params(self.pgp, self.gop, self.gep, self.rounds, self.lfactor_q16,
                           self.sfactor_q16, self.minfactor_q16, self.mode, None)
        keep = None
        if self.matrix is not None:
            keep = np.ascontiguousarray(self.matrix, dtype=np.int8)
            assert keep.shape == (24, 24)
            p.matrix = keep.ctypes.data_as(C.POINTER(C.c_int8))
        return p, keep


def encode(text: str) -> np.ndarray:
    b = text.encode("ascii")
    out = np.zeros(len(b), np.uint8)
    check(lib().hs_encode(b, len(b), out.ctypes.data), "hs_encode")
    return out


def builtin_matrix() -> np.ndarray:
    out = np.zeros((24, 24), np.int8)
    check(lib().hs_builtin_matrix(out.ctypes.data), "hs_builtin_matrix")
    return out


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream   # torch.cuda.Stream


class Database:
    """A database resident on the current CUDA device (hs_db_load).  With
    index_base > 0 it is a shard whose first sequence has that global index
    (hs_db_load_shard): hits report, and draws use, global indices."""

    def __init__(self, codes, offsets, stream=None, index_base: int = 0):
        codes = np.ascontiguousarray(codes, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        h = C.c_void_p()
        check(lib().hs_db_load_shard(codes.ctypes.data if len(codes) else None, offsets.ctypes.data,
                                     len(offsets) - 1, index_base, _stream_ptr(stream), C.byref(h)),
              "hs_db_load_shard")
        self.index_base = index_base
        self._h = h
        n, r, m = C.c_int64(), C.c_int64(), C.c_int32()
        check(lib().hs_db_info(h, C.byref(n), C.byref(r), C.byref(m)), "hs_db_info")
        self.n, self.residues, self.max_len = n.value, r.value, m.value

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("database closed")
        return self._h

    SCHEDULE_LENGTH, SCHEDULE_INPUT = 0, 1

    def set_schedule(self, schedule: int, stream=None):
        """Scan order: SCHEDULE_LENGTH (longest first, the default) or
        SCHEDULE_INPUT (database order).  Results do not depend on it."""
        check(lib().hs_db_set_schedule(self.handle, schedule, _stream_ptr(stream)), "hs_db_set_schedule")

    def schedule(self):
        """(order, cumres): database index at each scan position and the
        residues before each position (hs_db_get_schedule)."""
        order = np.zeros(max(self.n, 1), np.int32)
        cumres = np.zeros(self.n + 1, np.int64)
        check(lib().hs_db_get_schedule(self.handle, order.ctypes.data, cumres.ctypes.data), "hs_db_get_schedule")
        return order[: self.n], cumres

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().hs_db_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def workspace_size(db: Database, qlen: int, k: int) -> int:
    b = C.c_size_t()
    check(lib().hs_search_workspace_size(db.handle, qlen, k, C.byref(b)), "hs_search_workspace_size")
    return b.value


def search(db: Database, query, k: int, params: Params | None = None, seed: int = 0, stream=None):
    """hs_search: host query in, (hits structured array, ops uint32 array) out."""
    q = np.ascontiguousarray(query, dtype=np.uint8)
    p, _keep = (params or Params()).to_c()
    nh = min(k, db.n)
    hits = np.zeros(max(nh, 1), HIT_DTYPE)
    cap = lib().hs_ops_capacity(len(q), k)
    ops = np.zeros(max(cap, 1), np.uint32)
    n_out, used = C.c_int32(), C.c_int64()
    check(lib().hs_search(db.handle, q.ctypes.data, len(q), C.byref(p), k, seed & (2**64 - 1),
                          _stream_ptr(stream), hits.ctypes.data, C.byref(n_out), ops.ctypes.data,
                          cap, C.byref(used)), "hs_search")
    return hits[:n_out.value].copy(), ops[:used.value].copy()


def search_threshold(db: Database, query, threshold: int, max_hits: int, params: Params | None = None,
                     seed: int = 0, stream=None):
    """hs_search_threshold: every pair scoring >= threshold (at most
    max_hits, ranked) -> (hits, ops, number of pairs at or above)."""
    q = np.ascontiguousarray(query, dtype=np.uint8)
    p, _keep = (params or Params()).to_c()
    nh = min(max_hits, db.n)
    hits = np.zeros(max(nh, 1), HIT_DTYPE)
    cap = lib().hs_ops_capacity(len(q), max_hits)
    ops = np.zeros(max(cap, 1), np.uint32)
    n_out, above, used = C.c_int32(), C.c_int64(), C.c_int64()
    check(lib().hs_search_threshold(db.handle, q.ctypes.data, len(q), C.byref(p), threshold, max_hits,
                                    seed & (2**64 - 1), _stream_ptr(stream), hits.ctypes.data, C.byref(n_out),
                                    C.byref(above), ops.ctypes.data, cap, C.byref(used)), "hs_search_threshold")
    return hits[:n_out.value].copy(), ops[:used.value].copy(), int(above.value)


def _tuning(tuning):
    if tuning is None:
        return None
    if isinstance(tuning, _lib.hs_batch_tuning):
        return tuning
    unknown = set(tuning) - set(TUNING_KEYS)
    if unknown:
        raise ValueError("unknown tuning keys: %s" % sorted(unknown))
    return _lib.hs_batch_tuning(*[int(tuning.get(key, 0)) for key in TUNING_KEYS])


TUNING_KEYS = ("chunks", "warps", "flat_min_chunks", "flat_max_iters", "long_len")


def _pack_queries(queries):
    qs = [np.ascontiguousarray(q, dtype=np.uint8) for q in queries]
    off = np.zeros(len(qs) + 1, np.int64)
    np.cumsum([len(q) for q in qs], out=off[1:])
    cat = np.concatenate(qs) if qs else np.zeros(0, np.uint8)
    return cat, off


def search_batch(db: Database, queries, k: int, params: Params | None = None, seeds=None, tuning=None,
                 stream=None):
    """hs_search_batch: many queries in one scan launch.  Returns a list of
    (hits, ops) per query, each exactly what search() gives for that query
    and its seed (seeds default to 0).  tuning: a dict with any of
    TUNING_KEYS (hs_batch_tuning; absent or 0 = the default)."""
    cat, off = _pack_queries(queries)
    nq = len(off) - 1
    sd = np.zeros(nq, np.uint64) if seeds is None else np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    p, _keep = (params or Params()).to_c()
    hits = np.zeros(max(nq * k, 1), HIT_DTYPE)
    cap = lib().hs_batch_ops_capacity(nq, int(off[-1]), k)
    ops = np.zeros(max(cap, 1), np.uint32)
    n_out, used = C.c_int32(), C.c_int64()
    t = _tuning(tuning)
    check(lib().hs_search_batch(db.handle, nq, cat.ctypes.data, off.ctypes.data, sd.ctypes.data, C.byref(p), k,
                                C.byref(t) if t is not None else None, _stream_ptr(stream), hits.ctypes.data,
                                C.byref(n_out), ops.ctypes.data, cap, C.byref(used)), "hs_search_batch")
    nh = n_out.value
    out = []
    for i in range(nq):
        h = hits[i * k:i * k + nh].copy()
        segs = [ops[x["ops_offset"]:x["ops_offset"] + x["ops_len"]] for x in h]
        o = np.concatenate(segs).astype(np.uint32) if segs else np.zeros(0, np.uint32)
        pos = 0
        for j in range(len(h)):
            h[j]["ops_offset"] = pos
            pos += h[j]["ops_len"]
        out.append((h, o))
    return out


def search_batch_device(db: Database, queries_cat, qoffsets, seeds, max_qlen: int, k: int,
                        params: Params | None = None, tuning=None, stream=None, workspace=None, out=None):
    """hs_search_batch_device with torch CUDA tensors (queries_cat uint8,
    qoffsets int64[nq+1], seeds int64/uint64[nq]); asynchronous."""
    import torch
    dev = queries_cat.device
    nq = int(qoffsets.numel()) - 1
    total = int(queries_cat.numel())
    b = C.c_size_t()
    check(lib().hs_search_batch_workspace_size(db.handle, nq, total, max_qlen, k, C.byref(b)),
          "hs_search_batch_workspace_size")
    if workspace is None or workspace.numel() < b.value:
        workspace = torch.empty(b.value, dtype=torch.uint8, device=dev)
    cap = lib().hs_batch_ops_capacity(nq, total, k)
    if out is None:
        out = {"hits": torch.empty(max(nq * k, 1) * HIT_DTYPE.itemsize, dtype=torch.uint8, device=dev),
               "ops": torch.empty(max(cap, 1), dtype=torch.int32, device=dev),
               "ops_used": torch.zeros(1, dtype=torch.int64, device=dev),
               "status": torch.zeros(1, dtype=torch.int32, device=dev)}
    out["workspace"] = workspace
    p, _keep = (params or Params()).to_c()
    t = _tuning(tuning)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    check(lib().hs_search_batch_device(db.handle, nq, queries_cat.data_ptr(), qoffsets.data_ptr(), seeds.data_ptr(),
                                       total, max_qlen, C.byref(p), k, C.byref(t) if t is not None else None,
                                       _stream_ptr(st), workspace.data_ptr(), b.value, out["hits"].data_ptr(),
                                       out["ops"].data_ptr(), cap, out["ops_used"].data_ptr(),
                                       out["status"].data_ptr()), "hs_search_batch_device")
    out["n_hits"] = min(k, db.n)
    out["nq"] = nq
    out["k"] = k
    return out


def search_device(db: Database, query, k: int, params: Params | None = None, seed: int = 0,
                  stream=None, workspace=None, want_scores: bool = False, want_cells: bool = False,
                  out=None):
    """hs_search_device with torch CUDA tensors; asynchronous on `stream`.

    query: uint8 CUDA tensor.  Returns a dict of CUDA tensors: hits (uint8
    bytes, view with HIT_DTYPE after copying), ops, ops_used, status and
    optionally scores / cells.  Pass `out` (a previous result) and
    `workspace` to reuse buffers."""
    import torch
    dev = query.device
    qlen = int(query.numel())
    nh = min(k, db.n)
    ws_bytes = workspace_size(db, qlen, k)
    if workspace is None or workspace.numel() < ws_bytes:
        workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    cap = lib().hs_ops_capacity(qlen, k)
    if out is None:
        out = {
            "hits": torch.empty(max(nh, 1) * HIT_DTYPE.itemsize, dtype=torch.uint8, device=dev),
            "ops": torch.empty(max(cap, 1), dtype=torch.int32, device=dev),
            "ops_used": torch.zeros(1, dtype=torch.int64, device=dev),
            "status": torch.zeros(1, dtype=torch.int32, device=dev),
        }
        if want_scores:
            out["scores"] = torch.empty(max(db.n, 1), dtype=torch.int32, device=dev)
        if want_cells:
            out["cells"] = torch.empty(max(db.n, 1), dtype=torch.int64, device=dev)
    out["workspace"] = workspace
    p, _keep = (params or Params()).to_c()
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    check(lib().hs_search_device(
        db.handle, query.data_ptr(), qlen, C.byref(p), k, seed & (2**64 - 1), _stream_ptr(st),
        workspace.data_ptr(), ws_bytes, out["hits"].data_ptr(), out["ops"].data_ptr(), cap,
        out["ops_used"].data_ptr(),
        out["scores"].data_ptr() if "scores" in out else None,
        out["cells"].data_ptr() if "cells" in out else None,
        out["status"].data_ptr()), "hs_search_device")
    out["n_hits"] = nh
    return out


def search_device_noalloc(db: Database, query, k: int, out, params: Params | None = None, seed: int = 0,
                          stream=None):
    """hs_search_device_noalloc: the device search for callers that cannot
    allocate device memory while searching.  `out` must hold preallocated
    CUDA tensors "hits", "ops", "ops_used", "status" (and optionally
    "scores", "cells"), e.g. a previous search_device result; nothing is
    allocated here.  Scratch is the library's fixed 8 MiB area."""
    import torch
    qlen = int(query.numel())
    p, _keep = (params or Params()).to_c()
    st = stream if stream is not None else torch.cuda.current_stream(query.device)
    check(lib().hs_search_device_noalloc(
        db.handle, query.data_ptr(), qlen, C.byref(p), k, seed & (2**64 - 1), _stream_ptr(st),
        out["hits"].data_ptr(), out["ops"].data_ptr(), int(out["ops"].numel()), out["ops_used"].data_ptr(),
        out["scores"].data_ptr() if "scores" in out else None,
        out["cells"].data_ptr() if "cells" in out else None,
        out["status"].data_ptr()), "hs_search_device_noalloc")
    out["n_hits"] = min(k, db.n)
    return out


def device_result_to_host(out):
    """Copies a search_device result back: (hits structured array, ops)."""
    st = int(out["status"].item())
    if st != 0:
        raise HsError(st, "hs_search_device (device status)")
    nh = out["n_hits"]
    hits = np.frombuffer(out["hits"].cpu().numpy().tobytes(), dtype=HIT_DTYPE)[:nh].copy()
    used = int(out["ops_used"].item()) if nh else 0
    ops = out["ops"][:used].cpu().numpy().view(np.uint32).copy()
    return hits, ops


def get_alignment(db: Database, query, db_index: int, params: Params | None = None, seed: int = 0,
                  stream=None):
    """hs_get_alignment: (score, ops, hit record) of one pair."""
    q = np.ascontiguousarray(query, dtype=np.uint8)
    p, _keep = (params or Params()).to_c()
    cap = 2 * len(q) + 4
    ops = np.zeros(cap, np.uint32)
    score, n = C.c_int32(), C.c_int64()
    hit = np.zeros(1, HIT_DTYPE)
    check(lib().hs_get_alignment(db.handle, q.ctypes.data, len(q), C.byref(p), seed & (2**64 - 1),
                                 db_index, _stream_ptr(stream), ops.ctypes.data, cap, C.byref(score),
                                 C.byref(n), hit.ctypes.data), "hs_get_alignment")
    return int(score.value), ops[:n.value].copy(), hit[0]


def ops_to_rows(ops, q, t):
    """Expands run-length ops into the two alignment rows (GAP = 255)."""
    rq, rt = [], []
    i = j = 0
    for v in np.asarray(ops, dtype=np.uint32):
        op, n = int(v) & 3, int(v) >> 2
        for _ in range(n):
            if op == HS_OP_M:
                rq.append(int(q[i])); rt.append(int(t[j])); i += 1; j += 1
            elif op == HS_OP_I:
                rq.append(int(q[i])); rt.append(GAP); i += 1
            elif op == HS_OP_D:
                rq.append(GAP); rt.append(int(t[j])); j += 1
            else:
                raise ValueError("bad op %d" % op)
    if i != len(q) or j != len(t):
        raise ValueError("ops do not cover both sequences")
    return np.array(rq, np.uint8), np.array(rt, np.uint8)
