"""CPU oracle for the heuristic database search of Nag & Karforma (arXiv 1508.06561).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code that may import this
package.  The product path (``paper_1508_06561_gb300``) never does, and the two
share no code: the oracle has its own alphabet, matrix parser, Philox generator
and algorithm, all in ``hs_oracle.c`` (plain C, compiled with gcc by
``build()``), following Fig. 1 and Sec. III.B of the paper step by step.

The heuristic's own choices (how long each piece is, which shift wins, what
each step lays out) are pinned by an independent step trace in the tests
(numpy's Philox, integer piece sizes, numpy sliding-window argmax), beside
the invariants (rescore, DP optimum bound, closed forms); the GPU path must
agree with the oracle bit for bit.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hs_oracle.c")
LIB = os.path.join(HERE, "libhs_oracle.so")
BLOSUM62_TXT = os.path.join(HERE, "blosum62.txt")

GAP = 0xFF
LETTERS = "ARNDCQEGHILKMFPSTWYVBZX*"
MODE_DB = 0
MODE_FULL = 1


def build(force: bool = False) -> str:
    """Compile hs_oracle.c into libhs_oracle.so next to it (gcc, -O2, no SIMD flags)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-Wall", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


class Params(C.Structure):
    """Algorithm parameters (Sec. III.B.1); factors in Q16 (65536 == 1.0)."""
    _fields_ = [("pgp", C.c_int32), ("gop", C.c_int32), ("gep", C.c_int32),
                ("rounds", C.c_int32), ("lfactor_q16", C.c_uint32),
                ("sfactor_q16", C.c_uint32), ("minfactor_q16", C.c_uint32),
                ("mode", C.c_int32)]


def paper_params(**kw) -> Params:
    """The parameter set of Sec. IV: PGP=0, GOP=10, GEP=5, LFactor=0.5,
    SFactor=1, MinFactor=0.5, and Rounds=1 for database search (Sec. III.B.3 a)."""
    d = dict(pgp=0, gop=10, gep=5, rounds=1, lfactor_q16=32768, sfactor_q16=65536,
             minfactor_q16=32768, mode=MODE_DB)
    d.update(kw)
    return Params(**d)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def load(path):
    """Loads a build of hs_oracle.c with the argument types declared (the
    tests also load copies with planted mistakes, to show the pins catch them)."""
    L = C.CDLL(path)
    P = C.POINTER
    u8p, i8p, i64p, u64p, i32p = P(C.c_uint8), P(C.c_int8), P(C.c_int64), P(C.c_uint64), P(C.c_int32)
    L.or_philox4x64_10.argtypes = [u64p, u64p, u64p]
    L.or_draw16.argtypes = [C.c_uint64] * 4
    L.or_draw16.restype = C.c_uint32
    L.or_encode.argtypes = [C.c_char_p, C.c_int64, u8p]
    L.or_parse_matrix.argtypes = [C.c_char_p, i8p]
    L.or_parse_matrix.restype = C.c_int
    L.or_score_rows.argtypes = [u8p, u8p, C.c_int64, i8p, C.c_int32, C.c_int32, C.c_int32, i64p]
    L.or_score_rows.restype = C.c_int
    L.or_best_shift.argtypes = [u8p, C.c_int64, u8p, C.c_int64, i8p, i64p]
    L.or_best_shift.restype = C.c_int64
    L.or_best_shift_full.argtypes = [u8p, C.c_int64, u8p, C.c_int64, i8p, i64p]
    L.or_best_shift_full.restype = C.c_int64
    L.or_align_pair.argtypes = [u8p, C.c_int64, u8p, C.c_int64, i8p, P(Params), C.c_uint64,
                                C.c_uint64, u8p, u8p, i64p, i32p, i64p]
    L.or_align_pair.restype = C.c_int64
    L.or_search_scores.argtypes = [u8p, i64p, i64p, C.c_int64, u8p, C.c_int64, i8p, P(Params),
                                   C.c_uint64, C.c_int32, i64p, i64p]
    L.or_search_scores.restype = C.c_int32
    L.or_topk.argtypes = [i64p, C.c_int64, C.c_int32, i64p]
    L.or_topk.restype = C.c_int32
    L.or_periphery_opt.argtypes = [u8p, C.c_int64, u8p, C.c_int64, i8p, C.c_int32, C.c_int32, C.c_int32]
    L.or_periphery_opt.restype = C.c_int64
    L.or_smith_waterman.argtypes = [u8p, C.c_int64, u8p, C.c_int64, i8p, C.c_int32, C.c_int32]
    L.or_smith_waterman.restype = C.c_int64
    return L


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _mat(M):
    M = np.ascontiguousarray(M, dtype=np.int8)
    assert M.shape == (24, 24)
    return M


def philox4x64_10(ctr, key):
    c = (C.c_uint64 * 4)(*[int(x) & (2**64 - 1) for x in ctr])
    k = (C.c_uint64 * 2)(*[int(x) & (2**64 - 1) for x in key])
    o = (C.c_uint64 * 4)()
    lib().or_philox4x64_10(c, k, o)
    return [int(x) for x in o]


def draw16(seed, d, r, i):
    return int(lib().or_draw16(seed, d, r, i))


def encode(s: str) -> np.ndarray:
    b = s.encode("ascii")
    out = np.zeros(len(b), dtype=np.uint8)
    lib().or_encode(b, len(b), _p(out, C.c_uint8))
    return out


def parse_matrix(text: str) -> np.ndarray:
    out = np.zeros((24, 24), dtype=np.int8)
    if lib().or_parse_matrix(text.encode("ascii"), _p(out, C.c_int8)) != 0:
        raise ValueError("malformed matrix text")
    return out


def blosum62() -> np.ndarray:
    with open(BLOSUM62_TXT) as f:
        return parse_matrix(f.read())


def score_rows(rq, rt, M, pgp, gop, gep) -> int:
    rq, rt, M = _u8(rq), _u8(rt), _mat(M)
    assert rq.shape == rt.shape
    s = C.c_int64()
    if lib().or_score_rows(_p(rq, C.c_uint8), _p(rt, C.c_uint8), len(rq), _p(M, C.c_int8),
                           pgp, gop, gep, C.byref(s)) != 0:
        raise ValueError("gap-gap column")
    return int(s.value)


def best_shift(large, small, M):
    """One database-mode getBestSubsequenceAlignment: returns (k*, V(k*))."""
    large, small, M = _u8(large), _u8(small), _mat(M)
    k = C.c_int64()
    v = lib().or_best_shift(_p(large, C.c_uint8), len(large), _p(small, C.c_uint8), len(small),
                            _p(M, C.c_int8), C.byref(k))
    return int(k.value), int(v)


def best_shift_full(large, small, M):
    """One full-slide getBestSubsequenceAlignment (shifts -(|small|-1) ..
    |large|-1, overlap only): returns (k*, V(k*))."""
    large, small, M = _u8(large), _u8(small), _mat(M)
    k = C.c_int64()
    v = lib().or_best_shift_full(_p(large, C.c_uint8), len(large), _p(small, C.c_uint8), len(small),
                                 _p(M, C.c_int8), C.byref(k))
    return int(k.value), int(v)


def align_pair(q, t, M, params: Params, seed: int, dbidx: int, using=None):
    """AlignSequences for one pair: (score, query_row, target_row, round, cells).
    using: another loaded build (load()) instead of this one."""
    q, t, M = _u8(q), _u8(t), _mat(M)
    cap = len(q) + len(t) + 1
    rq = np.zeros(cap, np.uint8)
    rt = np.zeros(cap, np.uint8)
    n = C.c_int64()
    r = C.c_int32()
    cells = C.c_int64()
    s = (using or lib()).or_align_pair(_p(q, C.c_uint8), len(q), _p(t, C.c_uint8), len(t), _p(M, C.c_int8),
                            C.byref(params), seed, dbidx, _p(rq, C.c_uint8), _p(rt, C.c_uint8),
                            C.byref(n), C.byref(r), C.byref(cells))
    return int(s), rq[:n.value].copy(), rt[:n.value].copy(), int(r.value), int(cells.value)


def search_scores(codes, offsets, q, M, params: Params, seed: int, idx=None, nthreads=None,
                  want_cells=True):
    """Scores (int64) of the query against targets idx (default: all).

    Returns (scores, cells or None, threads_used)."""
    codes = _u8(codes)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    q, M = _u8(q), _mat(M)
    n = len(offsets) - 1 if idx is None else len(idx)
    idxa = None if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
    scores = np.zeros(n, np.int64)
    cells = np.zeros(n, np.int64) if want_cells else None
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    used = lib().or_search_scores(
        _p(codes, C.c_uint8), _p(offsets, C.c_int64),
        None if idxa is None else _p(idxa, C.c_int64), n, _p(q, C.c_uint8), len(q),
        _p(M, C.c_int8), C.byref(params), seed, nthreads, _p(scores, C.c_int64),
        None if cells is None else _p(cells, C.c_int64))
    return scores, cells, int(used)


def topk(scores, k):
    scores = np.ascontiguousarray(scores, dtype=np.int64)
    out = np.zeros(max(k, 1), np.int64)
    m = lib().or_topk(_p(scores, C.c_int64), len(scores), k, _p(out, C.c_int64))
    return out[:m].copy()


def periphery_opt(x, y, M, pgp, gop, gep) -> int:
    x, y, M = _u8(x), _u8(y), _mat(M)
    return int(lib().or_periphery_opt(_p(x, C.c_uint8), len(x), _p(y, C.c_uint8), len(y),
                                      _p(M, C.c_int8), pgp, gop, gep))


def smith_waterman(x, y, M, gop, gep) -> int:
    x, y, M = _u8(x), _u8(y), _mat(M)
    return int(lib().or_smith_waterman(_p(x, C.c_uint8), len(x), _p(y, C.c_uint8), len(y),
                                       _p(M, C.c_int8), gop, gep))
