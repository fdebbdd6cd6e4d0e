"""Builds libhsearch.so (the CUDA kernels + C ABI) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_1508_06561_gb300/libhsearch.so`` with the CUDA runtime linked
statically, so the library needs nothing but the NVIDIA kernel driver at
run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libhsearch.so")
SOURCES = ["hs_api.cu", "hs_scan.cu", "hs_topk.cu", "hs_noalloc.cu", "hs_sort.cu"]
# the integer issue-rate microbenchmark behind the scan's roofline (its own library)
PEAK_LIB = os.path.join(PKG, "libhspeak.so")
PEAK_SOURCES = ["hs_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(ROOT, "include", "hsearch.h"))
    return out


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(PEAK_LIB):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(PEAK_LIB))
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                    "-I", os.path.join(ROOT, "include")] + (extra or [])
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES) + len(PEAK_SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES + PEAK_SOURCES))
    if verbose:
        for _, err in results:
            if err:
                print(err)
    objs = [o for o, _ in results]
    for lib, srcs, script in ((LIB, SOURCES, "exports.map"), (PEAK_LIB, PEAK_SOURCES, "peak_exports.map")):
        tmp = lib + ".tmp%d" % os.getpid()
        mine = [o for o in objs if os.path.basename(o)[:-2] + ".cu" in srcs]
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-Xlinker",
                                 "--version-script=" + os.path.join(CSRC, script), "-o", tmp] + mine
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
