"""The top-k kernel on the CPU, checked against a plain ranking.

csrc/hs_topk.cu's kernel (per-CTA slice selection by score histograms, the
last CTA's merge from one histogram of the candidates' scores, its radix
fallback, the bitonic sort) is cut out verbatim and compiled as plain C++
into tests/emu/topk_emu.cpp, which runs each CTA as 512 threads (warps in
lockstep, a CTA barrier) and the CTAs one after another.  The ranked
(index, score) list must equal numpy's ranking by score descending, then
index ascending (reading A10).
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1508_06561_gb300", "csrc")


def topk_source():
    with open(os.path.join(CSRC, "hs_topk.cu")) as f:
        s = f.read()
    a = s.find("namespace {")
    b = s.find("}  // namespace", a)
    assert a >= 0 and b > a and "topk_kernel(" in s[a:b], "top-k markers not found in hs_topk.cu"
    return s[a:b + len("}  // namespace")] + "\n"


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("topk_emu")
    with open(d / "hs_topk_region.inc", "w") as f:
        f.write(topk_source())
    exe = str(d / "topk_emu")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-pthread", "-Wno-unknown-pragmas",
                           "-I", os.path.join(ROOT, "tests", "emu"), "-I", str(d), "-I", CSRC,
                           "-I", os.path.join(ROOT, "include"), "-o", exe,
                           os.path.join(ROOT, "tests", "emu", "topk_emu.cpp")])
    return exe, d


def run(emu, scores, k, ctas):
    exe, d = emu
    n = len(scores)
    inp, out = str(d / "in.bin"), str(d / "out.bin")
    with open(inp, "wb") as f:
        f.write(struct.pack("<qii", n, k, ctas))
        f.write(np.ascontiguousarray(scores, np.int32).tobytes())
    subprocess.run([exe, inp, out], check=True, timeout=600)
    with open(out, "rb") as f:
        b = f.read()
    nh = min(k, n)
    return np.frombuffer(b, np.int64, nh), np.frombuffer(b, np.int32, nh, 8 * nh)


def ranked(scores, k):
    idx = np.lexsort((np.arange(len(scores)), -scores.astype(np.int64)))[:min(k, len(scores))]
    return idx, scores[idx]


@pytest.mark.parametrize("n,k,ctas,lo,hi", [
    (5000, 10, 4, -100, 200),                  # narrow range: histogram merge
    (20000, 100, 8, -2000, 2000),
    (50000, 1000, 6, -10**6, 10**6),           # candidates span >= 4096 scores: radix merge
    (3000, 100, 3, 0, 3),                      # ties everywhere: lowest indices win
    (12000, 700, 8, 5, 6),                     # one score: more than 4096 candidates tie
    (100, 100, 4, -5, 5),                      # k = n
    (7, 10, 4, 0, 10),                         # k > n, empty slices
    (1, 5, 2, 0, 1),
])
def test_ranking_matches(emu, n, k, ctas, lo, hi):
    rng = np.random.default_rng(n + k)
    s = rng.integers(lo, hi, n).astype(np.int32)
    got_i, got_s = run(emu, s, k, ctas)
    want_i, want_s = ranked(s, k)
    assert np.array_equal(got_i, want_i) and np.array_equal(got_s, want_s)


def test_extreme_scores(emu):
    s = np.array([np.iinfo(np.int32).min + 1, np.iinfo(np.int32).max, 0, -1, 1, np.iinfo(np.int32).max], np.int32)
    got_i, got_s = run(emu, s, 4, 3)
    want_i, want_s = ranked(s, 4)
    assert np.array_equal(got_i, want_i) and np.array_equal(got_s, want_s)
