"""Build ``libaesgb.so`` in-tree: every ``csrc/*.cu`` and ``csrc/*.cpp`` compiled
in parallel with nvcc for sm_103a only, then linked into one shared library
with the CUDA runtime linked statically.

``python -m paper_1902_05234_gb300.build`` (or ``__graft_entry__.build()``)
runs it; objects go to ``_build/`` next to this file.  A rebuild happens only
when a source or header is newer than the library.

``build(debug=True)`` (``--debug``) makes ``libaesgb_debug.so`` from the same
sources with AESGB_BOUNDS_CHECK defined: every shared-memory table, tile,
mask and key-slot access and the batch and TMA kernels' global ranges are
checked, a failed check is counted (``aes_debug_bounds_violations``) and its
access skipped.  Objects go to ``_build_debug/``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libaesgb.so")
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(PKG, "libaesgb_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libaesgb.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _inputs():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) \
        + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def _compile(src: str, nvcc: str, debug: bool = False) -> str:
    obj = os.path.join(BUILD_DEBUG if debug else BUILD, os.path.basename(src) + ".o")
    cmd = [nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O2",
           "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
    if debug:
        cmd[1:1] = ["-DAESGB_BOUNDS_CHECK"]
    elif src.endswith(".cu"):
        # every nvcc/cudafe/ptxas warning is an error: a host-only helper called
        # from device code is only a warning otherwise, and the kernel then
        # silently compiles to nothing.  The bitsliced kernel (ct.cu) keeps 128
        # plane registers per thread and runs at the 255-register limit with a
        # few bytes of spill by design, so only it is exempt from the spill check.
        cmd[1:1] = ["--Werror", "all-warnings"]
        if os.path.basename(src) != "ct.cu":
            cmd[1:1] = ["-Xptxas", "-warn-spills"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(debug):
        return lib
    nvcc = _nvcc()
    os.makedirs(BUILD_DEBUG if debug else BUILD, exist_ok=True)
    srcs = _sources()
    workers = max(1, min(len(srcs), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(lambda s: _compile(s, nvcc, debug), srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static", "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}")
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv)
