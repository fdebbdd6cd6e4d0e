"""The batched scan's work loop on the CPU, checked against the oracle.

batch_items -- (query, chunk) items from one counter, the per-item role
split of a length-ordered chunk (a binary search for the first target
shorter than the query), one role profile staged at a time, a CTA-shared
position counter per sub-range, per-query lengths and seeds -- and the pair
loop it runs are cut verbatim out of csrc/hs_scan.cu and compiled as plain
C++ into tests/emu/batch_emu.cpp: several CTAs of lockstep warps at once,
each with its own barrier, staged profile and slots.  Every query's scores
must equal the oracle's for that query alone.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1508_06561_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1508_06561_gb300", "csrc")


def regions():
    with open(os.path.join(CSRC, "hs_scan.cu")) as f:
        s = f.read()
    a = s.find("constexpr int kLocalIters")
    b = s.find("// Plain scan: a persistent grid over one queue")
    assert a >= 0 and b > a, "pair-loop markers not found in hs_scan.cu"
    pairs = s[a:s.rfind("// ----", 0, b)]
    a = s.find("struct BatchScan {")
    b = s.find("__global__ void __launch_bounds__(kWarpsPerCta * 32, 3)\nscan_batch_kernel")
    assert a >= 0 and b > a, "batch-loop markers not found in hs_scan.cu"
    b = s.rfind("template <", 0, b)
    batch = s[a:b]
    assert "void batch_items(" in batch
    return pairs, batch


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("batch_emu")
    pairs, batch = regions()
    (d / "hs_pairs_region.inc").write_text(pairs)
    (d / "hs_batch_region.inc").write_text(batch)
    exe = str(d / "batch_emu")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-pthread", "-Wno-unknown-pragmas",
                           "-I", os.path.join(ROOT, "tests", "emu"), "-I", str(d), "-I", CSRC,
                           "-I", os.path.join(ROOT, "include"), "-o", exe,
                           os.path.join(ROOT, "tests", "emu", "batch_emu.cpp")])
    return exe, d


def run(emu, db, qs, seeds, M, p, ctas, warps, nchunk, chunk_step, smem):
    exe, d = emu
    qoff = np.zeros(len(qs) + 1, np.int64)
    np.cumsum([len(q) for q in qs], out=qoff[1:])
    hdr = struct.pack("<qqiiiiiiiiiiIII", db.n, len(db.codes), len(qs), ctas, warps, nchunk, chunk_step, smem,
                      p.pgp, p.gop, p.gep, p.rounds, p.lfactor_q16, p.sfactor_q16, p.minfactor_q16)
    inp, out = str(d / "in.bin"), str(d / "out.bin")
    with open(inp, "wb") as f:
        f.write(hdr)
        f.write(np.ascontiguousarray(M, np.int8).tobytes())
        f.write(np.ascontiguousarray(db.codes, np.uint8).tobytes())
        f.write(np.ascontiguousarray(db.offsets, np.int64).tobytes())
        f.write(qoff.tobytes())
        f.write(np.asarray(seeds, np.uint64).tobytes())
        f.write(np.concatenate(qs).astype(np.uint8).tobytes())
    subprocess.run([exe, inp, out], check=True, timeout=900)
    with open(out, "rb") as f:
        return np.frombuffer(f.read(), np.int32).reshape(len(qs), db.n)


@pytest.mark.parametrize("smem,chunk_step,nchunk", [(1, 1, 7), (1, 3, 8), (0, 1, 5)])
def test_batch_scores_equal_each_query_alone(emu, smem, chunk_step, nchunk):
    """smem 1: length order, each chunk's two roles as sub-ranges with their
    profile staged (wide CTAs take chunk_step chunks per item); smem 0:
    database order, both profiles read in place."""
    rng = np.random.default_rng(5 + 10 * smem + chunk_step)
    lengths = np.concatenate([rng.integers(1, 500, 120), [0, 1], [2100, 2600]])
    rng.shuffle(lengths)
    db = synth.db_from_lengths(rng, lengths)
    qs = [synth.residues(rng, L) for L in (1, 40, 150, 300, 700)]
    seeds = [11, 12, 13, 14, 15]
    M, p = O.blosum62(), O.paper_params()
    got = run(emu, db, qs, seeds, M, p, ctas=2, warps=2, nchunk=nchunk, chunk_step=chunk_step, smem=smem)
    for i, q in enumerate(qs):
        want = O.search_scores(db.codes, db.offsets, q, M, p, seeds[i])[0]
        bad = np.nonzero(got[i] != want)[0]
        assert bad.size == 0, "query %d differs at %s" % (i, bad[:5])
