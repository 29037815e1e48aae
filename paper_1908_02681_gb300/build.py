"""In-tree build of libpcr.so (nvcc, sm_103a only)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_PATH = os.path.join(HERE, "libpcr.so")
CEILINGS_PATH = os.path.join(HERE, "libpcr_ceilings.so")
SOURCES = ["pcr_api.cu"]
CEILING_SOURCES = ["ceilings.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

# -fmad=false: no implicit contraction anywhere; every fused multiply-add in the kernels is written out.
NVCC_FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-fmad=false",
              "-Xcompiler", "-fPIC", "-shared", "-Xptxas", "-warn-spills"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h", ".inc"))]
    return files + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]


def stale(path: str = LIB_PATH) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(f) > t for f in _inputs())


def _nvcc(sources, out, verbose):
    tmp = out + ".tmp"
    cmd = [NVCC, *NVCC_FLAGS, "-I", INCLUDE, "-I", CSRC, *[os.path.join(CSRC, s) for s in sources], "-o", tmp]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the rasterizer into libpcr.so next to this file (skipped when up to date)."""
    if not force and not stale(LIB_PATH):
        return LIB_PATH
    return _nvcc(SOURCES, LIB_PATH, verbose)


def build_ceilings(force: bool = False, verbose: bool = False) -> str:
    """Compile the roofline probes into libpcr_ceilings.so."""
    if not force and not stale(CEILINGS_PATH):
        return CEILINGS_PATH
    return _nvcc(CEILING_SOURCES, CEILINGS_PATH, verbose)


if __name__ == "__main__":
    build(force=True, verbose=True)
    build_ceilings(force=True, verbose=True)
