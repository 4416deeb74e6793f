"""Builds the CUDA library (libgsp.so) in-tree with nvcc for sm_103a.

Translation units compile in parallel, then link into one shared library that exports the C ABI
of include/gsp.h. Output: paper_1505_06022_gb300/_build/libgsp.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libgsp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["capi.cu", "sppm.cu", "scan_sort.cu", "grid_static.cu", "lbvh.cu", "membench.cu", "bvh_build.cpp"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _flags():
    # GSP_NVCC_EXTRA: extra nvcc arguments, e.g. -DGSP_PATH_MIN_BLOCKS=8 to sweep launch shapes
    extra = os.environ.get("GSP_NVCC_EXTRA", "").split()
    # -fmad=false: device arithmetic rounds as written (fused multiply-adds only where the source
    # spells them out), so one device function gives identical bits in every kernel it is inlined in
    return ARCH + ["-O3", "-fmad=false", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC] + extra


def _digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)) + ["../../include/gsp.h"]:
        path = os.path.join(CSRC, name)
        if os.path.isfile(path):
            h.update(name.encode())
            h.update(open(path, "rb").read())
    h.update(" ".join(_flags()).encode())
    return h.hexdigest()


# Everything the closest-hit kernel (k_trace, k_refine) is compiled from: a change elsewhere in the
# library leaves its profile counters valid.
TRACE_SOURCES = ["capi.cu", "devcommon.cuh", "launch.h", "persist.cuh", "gsp_internal.h"]


def trace_digest() -> str:
    """Digest of the closest-hit kernel's sources and compile flags. Include directories are left
    out: they are absolute paths, which differ between checkouts of the same sources."""
    h = hashlib.sha256()
    for name in TRACE_SOURCES:
        h.update(name.encode())
        h.update(open(os.path.join(CSRC, name), "rb").read())
    h.update(" ".join(f for f in _flags() if not os.path.isabs(f)).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "libgsp.sha256")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + _flags() + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
