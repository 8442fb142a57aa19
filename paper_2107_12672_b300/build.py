"""Build the renderer's CUDA library in-tree for B300 (sm_103a).

    python -m paper_2107_12672_b300.build [--force] [--verbose]

Compiles every csrc/*.cu with nvcc into _build/ and links
paper_2107_12672_b300/_lib/libdvr.so (static CUDA runtime, C ABI of
include/dvr.h). Rebuilds only what changed (sources or headers newer than
the objects). With --bounds it builds the bounds-checked library instead
(DVR_DEBUG_BOUNDS: every kernel index checked against its extent, failures
reported by the entry points), _lib/libdvr_bounds.so, from objects in
_build/bounds/.
"""
from __future__ import annotations

import argparse
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
BUILD = os.path.join(ROOT, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libdvr.so")
BOUNDS_LIB = os.path.join(LIBDIR, "libdvr_bounds.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                     "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _compile(src: str, verbose: bool, force: bool, bounds: bool = False) -> str:
    obj = os.path.join(BUILD, "bounds" if bounds else "", os.path.basename(src) + ".o")
    newest = max(os.path.getmtime(p) for p in [src, *_headers()])
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= newest:
        return obj
    cmd = [nvcc(), *NVCC_FLAGS, *(["-DDVR_DEBUG_BOUNDS"] if bounds else []), "-c", src, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
    if verbose:
        sys.stderr.write(res.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Compile and link libdvr.so (or, with bounds, libdvr_bounds.so);
    returns its path."""
    lib = BOUNDS_LIB if bounds else LIB
    os.makedirs(os.path.join(BUILD, "bounds") if bounds else BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, force, bounds), srcs))
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true", help="print ptxas register/smem usage")
    ap.add_argument("--bounds", action="store_true", help="the bounds-checked library (DVR_DEBUG_BOUNDS)")
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.verbose, bounds=a.bounds))
