"""Builds libvpgs.so in-tree for sm_103a with nvcc (no cmake, no torch extension).

Each CUDA translation unit is compiled in parallel into _build/, then linked
with the static CUDA runtime into paper_2505_18992_gb300/libvpgs.so.  A unit is
rebuilt when it or any header is newer than its object, or when the flags it
was compiled with (VPGS_NVCC_FLAGS included) have changed.
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
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libvpgs.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))


def _env_flags():
    """Extra nvcc flags from VPGS_NVCC_FLAGS (e.g. -DVPGS_PIX=2 to retune the compositing geometry)."""
    return os.environ.get("VPGS_NVCC_FLAGS", "").split()


def _compile(src: str, extra) -> str:
    """Compiles src unless its object is newer than every source and header and
    was built with the same flags (VPGS_NVCC_FLAGS included: the stamp file
    beside the object records them)."""
    obj = os.path.join(BUILD, os.path.basename(src).replace(".cu", ".o"))
    stamp = obj + ".flags"
    flags = [*ARCH, *NVCC_FLAGS, *_env_flags(), *extra]
    key = "\n".join(flags)
    newest = max([os.path.getmtime(src)] + [os.path.getmtime(h) for h in _headers()])
    same_flags = os.path.exists(stamp) and open(stamp).read() == key
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest and same_flags and not extra:
        return obj
    cmd = [nvcc(), *flags, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{res.stderr}")
    if extra and res.stderr:
        sys.stderr.write(res.stderr)
    with open(stamp, "w") as fh:
        fh.write(key)
    return obj


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every CUDA unit and link libvpgs.so; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < newest or extra:
        cmd = [nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-cudart", "static"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stderr}")
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="-v" in sys.argv)
