"""The C ABI library builds, loads and exports every declared entry point;
host-only entry points (no GPU needed) agree with the oracle's independent
tables, and argument checks fail before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_1508_06561_gb300 as P
from paper_1508_06561_gb300 import _lib, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "hsearch.h")


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hs_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["hs_db_load", "hs_search", "hs_search_device", "hs_get_alignment", "hs_db_free",
                 "hs_strerror", "hs_encode"]:
        assert must in names


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_exports_are_exactly_the_header(L):
    """The shared library's dynamic symbol table holds the C ABI and nothing
    else (internal C++ symbols stay local)."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if not nm:
        pytest.skip("nm not available")
    from paper_1508_06561_gb300 import build
    out = subprocess.run([nm, "-D", "--defined-only", build.LIB], capture_output=True, text=True, check=True).stdout
    exported = sorted({line.split()[-1] for line in out.splitlines() if line.split()[1:2] and line.split()[1] in "TW"})
    assert exported == declared_functions()


def test_builtin_matrix_equals_oracle_table(L):
    assert np.array_equal(P.builtin_matrix(), O.blosum62())


def test_encode_equals_oracle_encode(L):
    s = "ARNDCQEGHILKMFPSTWYVBZX*arndcqeghilkmfpstwyvbzxJOU1- "
    assert np.array_equal(P.encode(s), O.encode(s))


def test_params_check(L):
    p = _lib.hs_params()
    L.hs_params_default(C.byref(p))
    assert (p.pgp, p.gop, p.gep, p.rounds) == (0, 10, 5, 1)
    assert (p.lfactor_q16, p.sfactor_q16, p.minfactor_q16) == (32768, 65536, 32768)
    assert L.hs_params_check(C.byref(p)) == 0
    for field, bad in [("pgp", -1), ("gop", 1001), ("rounds", 0), ("lfactor_q16", 65537), ("mode", 3)]:
        q = _lib.hs_params()
        L.hs_params_default(C.byref(q))
        setattr(q, field, bad)
        assert L.hs_params_check(C.byref(q)) == _lib.HS_EINVAL, field
    M = O.blosum62().copy()
    M[0, 1] = 3                       # asymmetric
    q, keep = P.Params(matrix=M).to_c()
    assert L.hs_params_check(C.byref(q)) == _lib.HS_EINVAL


def test_strerror(L):
    for s in range(8):
        assert len(L.hs_strerror(s)) > 0


def test_db_load_rejects_bad_input_before_device_work(L):
    h = C.c_void_p()
    codes = np.zeros(10, np.uint8)
    bad_off = np.array([0, 5, 3, 10], np.int64)          # decreasing
    assert L.hs_db_load(codes.ctypes.data, bad_off.ctypes.data, 3, None, C.byref(h)) == _lib.HS_EINVAL
    off = np.array([1, 5, 10], np.int64)                 # offsets[0] != 0
    assert L.hs_db_load(codes.ctypes.data, off.ctypes.data, 2, None, C.byref(h)) == _lib.HS_EINVAL
    codes2 = np.array([0, 1, 24], np.uint8)              # code out of range
    off2 = np.array([0, 3], np.int64)
    assert L.hs_db_load(codes2.ctypes.data, off2.ctypes.data, 1, None, C.byref(h)) == _lib.HS_EINVAL
    off3 = np.array([0, 1_000_001], np.int64)            # too long
    big = np.zeros(1_000_001, np.uint8)
    assert L.hs_db_load(big.ctypes.data, off3.ctypes.data, 1, None, C.byref(h)) == _lib.HS_ETOOLONG


def test_ops_to_rows_roundtrip():
    q = np.array([1, 2, 3], np.uint8)
    t = np.array([4, 5], np.uint8)
    ops = np.array([(1 << 2) | 0, (2 << 2) | 1, (1 << 2) | 2], np.uint32)   # M, I I, D
    rq, rt = P.ops_to_rows(ops, q, t)
    assert rq.tolist() == [1, 2, 3, 255] and rt.tolist() == [4, 255, 255, 5]
    with pytest.raises(ValueError):
        P.ops_to_rows(ops[:2], q, t)


def test_peak_library_exports_exactly_its_header():
    """The integer issue-rate microbenchmark (the scan roofline's peak) is
    its own library; it exports include/hspeak.h's functions and nothing else."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if not nm:
        pytest.skip("nm not available")
    build.build()
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(os.path.dirname(HEADER), "hspeak.h")).read(), flags=re.S)
    declared = sorted(set(re.findall(r"\b(hsp_[a-z_0-9]+)\s*\(", text)))
    out = subprocess.run([nm, "-D", "--defined-only", build.PEAK_LIB], capture_output=True, text=True, check=True).stdout
    exported = sorted({line.split()[-1] for line in out.splitlines() if line.split()[1:2] and line.split()[1] in "TW"})
    assert exported == declared == ["hsp_measure", "hsp_ops_per_thread_trip"]
