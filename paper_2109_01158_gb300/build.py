"""Build libfemenergy.so in-tree for sm_103a (GB300) with nvcc.

Each translation unit under ``csrc/`` is compiled in parallel to an object file, then
linked into ``paper_2109_01158_gb300/libfemenergy.so``.  Run as a script or call
``build()``; objects are rebuilt only when a source or header is newer.  ``build(bounds=True)``
builds the bounds-checking variant (-DFE_DEBUG_BOUNDS) into ``libfemenergy_bounds.so`` from
objects of its own.
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
OBJDIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfemenergy.so")
BOUNDS_OBJDIR = os.path.join(PKG, "_build_bounds")
BOUNDS_LIB = os.path.join(PKG, "libfemenergy_bounds.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfemenergy.so")
    return exe


def _deps_mtime() -> float:
    files = (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
             + glob.glob(os.path.join(INCLUDE, "*.h")))
    return max((os.path.getmtime(f) for f in files), default=0.0)


def _compile(src: str, extra: list[str], objdir: str = OBJDIR) -> str:
    obj = os.path.join(objdir, os.path.basename(src).replace(".cu", ".o"))
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), _deps_mtime()):
        return obj
    cmd = [nvcc()] + ARCH + CFLAGS + extra + ["-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return obj


def build(verbose: bool = False, extra: list[str] | None = None, bounds: bool = False) -> str:
    """Compile every CUDA source and link the shared library; returns its path.  With
    bounds=True, the bounds-checking variant (objects and library of its own)."""
    objdir, lib = (BOUNDS_OBJDIR, BOUNDS_LIB) if bounds else (OBJDIR, LIB)
    os.makedirs(objdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    extra = list(extra or []) + (["-DFE_DEBUG_BOUNDS"] if bounds else [])
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, objdir), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, lib)
    if verbose:
        print(lib)
    return lib


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
