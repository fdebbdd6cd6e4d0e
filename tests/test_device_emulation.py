"""The scan's per-lane arithmetic, compiled for the host and run on the CPU.

tests/emu/lane_emu.cpp includes the kernel header (csrc/hs_device.cuh) with a
stub cuda_runtime.h and checks, for random inputs, that every packed 4-shift
chunk sum (byte lanes, widening every `flush` cells, masked edges, random
iteration segments) and every lane-local step equals the naive sum of matrix
entries, with the profile and target buffers placed against guard pages so
that any out-of-range read faults.  Matrix ranges cover BLOSUM62's, a wide
one (widen every 2 cells), the full int8 range (every cell) and a constant.
Two of the runs are repeated with AddressSanitizer and UBSan.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("emu") / "lane_emu")
    subprocess.check_call([gxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "tests", "emu"),
                           "-I", os.path.join(ROOT, "paper_1508_06561_gb300", "csrc"),
                           "-I", os.path.join(ROOT, "include"), "-o", exe,
                           os.path.join(ROOT, "tests", "emu", "lane_emu.cpp")])
    return exe


@pytest.mark.parametrize("seed,lo,hi", [(1, -4, 11), (2, -40, 50), (3, -128, 127), (4, 0, 0), (5, -1, 1)])
def test_lane_arithmetic_matches_naive_sums(emu, seed, lo, hi):
    r = subprocess.run([emu, str(seed), str(lo), str(hi)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "emu ok" in r.stdout


@pytest.fixture(scope="module")
def emu_sanitized(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("emu_san") / "lane_emu")
    r = subprocess.run([gxx, "-O1", "-g", "-std=c++17", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=undefined", "-Wno-unknown-pragmas",
                        "-I", os.path.join(ROOT, "tests", "emu"),
                        "-I", os.path.join(ROOT, "paper_1508_06561_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), "-o", exe,
                        os.path.join(ROOT, "tests", "emu", "lane_emu.cpp")], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("no sanitizer runtime: " + r.stderr[-200:])
    return exe


@pytest.mark.parametrize("seed,lo,hi", [(1, -4, 11), (3, -128, 127)])
def test_lane_arithmetic_is_free_of_undefined_behaviour(emu_sanitized, seed, lo, hi):
    """The same checks built with AddressSanitizer and UBSan (shifts past the
    word, signed overflow, out-of-bounds reads all abort the run)."""
    r = subprocess.run([emu_sanitized, str(seed), str(lo), str(hi)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "emu ok" in r.stdout
