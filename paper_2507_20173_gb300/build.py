"""Build libfsb.so in-tree for GB300 (sm_103a) with nvcc.

Every translation unit is compiled in parallel with one -gencode
(compute_103a -> sm_103a).  The per-fish arithmetic keeps IEEE semantics:
no --use_fast_math, no FMA contraction (--fmad=false), subnormals kept
(-ftz=false), correctly rounded division and square root.
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfsb.so")
# the debug library: the same sources with run-time invariant checks
# (-DFSB_DEBUG_BOUNDS, fsb_check.cuh), built beside the release one
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libfsb_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--fmad=false", "-ftz=false",
              "-prec-div=true", "-prec-sqrt=true", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-Wall", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found; the CUDA 13 toolkit is required")
    return exe


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cpp")))


def _headers() -> list[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs + [os.path.join(ROOT, "include", f)
                 for f in os.listdir(os.path.join(ROOT, "include"))]


def _compile(src: str, extra: list[str], out_dir: str = BUILD) -> tuple[str, str]:
    obj = os.path.join(out_dir, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc(), "-x", "cu", *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), proc.stderr))
    return obj, proc.stderr


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          debug: bool = False) -> str:
    """Compile every CUDA/C++ source of the library and link libfsb.so (or,
    with debug, libfsb_debug.so with the run-time invariant checks)."""
    out_dir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    flags = list(extra or []) + (["-DFSB_DEBUG_BOUNDS"] if debug else [])
    os.makedirs(out_dir, exist_ok=True)
    srcs = sources()
    newest = max(os.path.getmtime(p) for p in srcs + _headers())
    if not force and not extra and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        done = list(ex.map(lambda s: _compile(s, flags, out_dir), srcs))
    objs = [obj for obj, _ in done]
    if verbose:  # compiler remarks, e.g. ptxas -v register and spill counts
        for obj, log in done:
            if log.strip():
                print("== %s\n%s" % (os.path.basename(obj), log.rstrip()), file=sys.stderr)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcuda"]
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), proc.stderr))
    os.replace(tmp, lib)
    if verbose:
        print("built", lib, file=sys.stderr)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None,
          debug="--debug" in sys.argv)
