"""Builds the CUDA library libvt.so in-tree for sm_103a (GB300).

Each translation unit compiles in its own nvcc process (in parallel); the
objects link into ``paper_2412_04514_gb300/_build/libvt.so`` (or the directory
named by ``VT_BUILD_DIR``). Only nvcc and a host C++ compiler are needed; no
cmake, no torch headers. ``VT_NVCC_FLAGS`` adds compiler flags, e.g.
``-DVT_CHECKS`` for the bounds-checked debug build.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
# VT_BUILD_DIR: another build directory (a debug build beside the regular one)
BUILD = os.environ.get("VT_BUILD_DIR") or os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libvt.so")
SOURCES = ["scan.cu", "grid.cu", "knn.cu", "clip_f32.cu", "clip_f64.cu", "clip_robust.cu", "emit.cu", "vt_api.cu", "grid_static.cu", "adjoint.cu", "tune.cu", "range.cu", "clip_big.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "vt.h"), __file__]
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile (if stale) and return the path of libvt.so."""
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input() and not extra
            and not os.environ.get("VT_NVCC_FLAGS")):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    extra = (extra or []) + os.environ.get("VT_NVCC_FLAGS", "").split()

    def one(src: str) -> str:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    verbose = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if verbose else None
    print(build(force=True, verbose=verbose, extra=extra))
