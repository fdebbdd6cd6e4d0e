"""The database-load kernels on the CPU (row a1: the longest-first schedule
and its residue prefix, built on the device).

tests/emu/sort_emu.cpp runs csrc/hs_sort.cu's device code, cut out as it
stands, one CTA at a time with 32-thread lockstep warps and a CTA barrier,
in build_schedule's launch order.  The order must be numpy's stable sort by
descending length (equal lengths keep database order) and the prefix
numpy's cumulative sum; the three-pass exclusive prefix is also checked
alone over several blocks.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from paper_1508_06561_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1508_06561_gb300", "csrc")


def sort_source():
    """hs_sort.cu's device code (the anonymous namespace), verbatim."""
    with open(os.path.join(CSRC, "hs_sort.cu")) as f:
        s = f.read()
    a = s.find("constexpr int kSortThreads")
    b = s.find("}  // namespace", a)
    assert a >= 0 and b > a, "markers not found in hs_sort.cu"
    region = s[a:b]
    assert "residue_prefix_kernel" in region and "radix_scatter_kernel" in region
    return region


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("sort_emu")
    with open(d / "hs_sort_region.inc", "w") as f:
        f.write(sort_source())
    exe = str(d / "sort_emu")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-pthread", "-Wno-unknown-pragmas",
                           "-I", os.path.join(ROOT, "tests", "emu"), "-I", str(d), "-I", CSRC,
                           "-I", os.path.join(ROOT, "include"), "-o", exe,
                           os.path.join(ROOT, "tests", "emu", "sort_emu.cpp")])
    return exe, d


def run_sort(emu, lengths):
    exe, d = emu
    off = synth.offsets_from_lengths(np.asarray(lengths, np.int64))
    n = len(off) - 1
    inp, out = str(d / "in.bin"), str(d / "out.bin")
    with open(inp, "wb") as f:
        f.write(struct.pack("<q", n))
        f.write(np.ascontiguousarray(off, np.int64).tobytes())
    subprocess.run([exe, "sort", inp, out], check=True, timeout=600)
    b = open(out, "rb").read()
    return np.frombuffer(b, np.int32, n), np.frombuffer(b, np.int64, n + 1, 4 * n)


@pytest.mark.parametrize("case", ["equal-lengths", "lognormal", "wide-keys"])
def test_schedule_is_the_stable_longest_first_order(emu, case):
    rng = np.random.default_rng({"equal-lengths": 1, "lognormal": 2, "wide-keys": 3}[case])
    if case == "equal-lengths":         # many ties: stability decides the order
        L = rng.integers(0, 6, 9000)
    elif case == "lognormal":
        L = synth.lognormal_lengths(rng, 20000, 300, 0.6, 1, 35000)
    else:                               # lengths spanning three 8-bit digits
        L = rng.integers(0, 1_000_000, 5000)
    order, cumres = run_sort(emu, L)
    want = np.argsort(-np.asarray(L, np.int64), kind="stable")
    assert np.array_equal(order, want)
    assert np.array_equal(cumres, np.concatenate([[0], np.cumsum(np.asarray(L, np.int64)[want])]))


def test_residue_prefix_over_several_blocks(emu):
    """Enough targets for the three-pass residue prefix to use several CTAs."""
    rng = np.random.default_rng(4)
    L = rng.integers(1, 3000, 40000)
    order, cumres = run_sort(emu, L)
    assert np.array_equal(cumres, np.concatenate([[0], np.cumsum(L[np.argsort(-L, kind="stable")])]))


@pytest.mark.parametrize("m", [1, 1000, 16384, 16385, 50000])
def test_exclusive_prefix_of_counts(emu, m):
    exe, d = emu
    a = np.random.default_rng(m).integers(0, 300, m).astype(np.uint32)
    inp, out = str(d / "scan_in.bin"), str(d / "scan_out.bin")
    with open(inp, "wb") as f:
        f.write(struct.pack("<q", m))
        f.write(a.tobytes())
    subprocess.run([exe, "scan", inp, out], check=True, timeout=600)
    got = np.frombuffer(open(out, "rb").read(), np.uint32, m)
    want = np.concatenate([[0], np.cumsum(a.astype(np.uint64))[:-1]]).astype(np.uint32)
    assert np.array_equal(got, want)
