"""Oracle for the point-cloud rasterizer (arXiv 1908.02681, Sections 2.1 and 2.2).

TEST INFRASTRUCTURE ONLY. The tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import it; the rendering library (`paper_1908_02681_gb300`) never does, and the two share no code.

This module is a thin ctypes wrapper around `pcr_oracle.cpp`, a plain single-threaded FP64 C++
implementation of the definition (per-point projection, 40-bit depth quantisation, key packing,
per-pixel minimum, resolve, and the high-quality splatting band test, sums and average). See the C++
file's header for the exact operation order and the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcr_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "libpcroracle.so")
_lib = None

EMPTY = 0xFFFFFFFFFFFFFFFF
Q_MAX = (1 << 40) - 2


def build(force: bool = False) -> str:
    """Compile the oracle in place: -O2, no floating-point contraction, no fast-math."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_P = ctypes.c_void_p
_VIEW_ARGS = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int, _P, ctypes.c_int,
              ctypes.c_int]


def _declare(lib):
    lib.oracle_project.argtypes = [_P, ctypes.c_uint64, _P] + _VIEW_ARGS + [_P, _P, _P]
    lib.oracle_render_atomicmin.argtypes = [_P, ctypes.c_uint64, _P] + _VIEW_ARGS + [_P]
    lib.oracle_clear.argtypes = [_P, ctypes.c_uint64]
    lib.oracle_clear.restype = None
    lib.oracle_hq_accumulate.argtypes = ([_P, ctypes.c_uint64, _P] + _VIEW_ARGS +
                                         [_P, ctypes.c_uint32, ctypes.c_uint32, _P, _P, _P, _P])
    lib.oracle_resolve_basic.argtypes = [_P, ctypes.c_uint64, ctypes.c_uint32, _P]
    lib.oracle_resolve_basic.restype = None
    lib.oracle_resolve_hq.argtypes = [_P, _P, _P, _P, ctypes.c_uint64, ctypes.c_uint32, _P]
    lib.oracle_resolve_hq.restype = None
    lib.oracle_bruteforce_pixel.argtypes = [_P, ctypes.c_uint64, _P] + _VIEW_ARGS + [ctypes.c_int, ctypes.c_int]
    lib.oracle_bruteforce_pixel.restype = ctypes.c_uint64
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def use_library(path: str | None):
    """Point this module at another build of the oracle source (the mutation tests compile copies of
    it with planted mistakes); None restores the default build."""
    global _lib
    _lib = None if path is None else _declare(ctypes.CDLL(path))


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile oracle source text (e.g. a mutated copy) to a shared library at out_path."""
    src = out_path + ".cpp"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           src, "-o", out_path])
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _pts(points) -> np.ndarray:
    a = np.ascontiguousarray(points)
    if a.dtype != np.uint32 or a.ndim != 2 or a.shape[1] != 4:
        raise ValueError("points must be an (n, 4) uint32 array (float32 x, y, z bits + RGBA8)")
    return a


class _ViewArgs:
    """Marshals a view (any object with view_proj, near, far, width, height, depth_mode, metric_scale
    and optional ranges) into the C argument list; keeps the arrays alive."""

    def __init__(self, view):
        self.M = np.ascontiguousarray(np.asarray(view.view_proj, dtype=np.float64).reshape(16))
        ranges = getattr(view, "ranges", None)
        self.ranges = None if ranges is None else np.ascontiguousarray(np.asarray(ranges, dtype=np.float64).reshape(-1, 3))
        n_ranges = 0 if self.ranges is None else self.ranges.shape[0]
        self.W, self.H = int(view.width), int(view.height)
        self.args = [float(view.near), float(view.far), int(getattr(view, "depth_mode", 0)),
                     float(getattr(view, "metric_scale", 1000.0)), n_ranges,
                     None if self.ranges is None else self.ranges.ctypes.data, self.W, self.H]


def project(points, view):
    """Per point: (pixel index py*W+px or -1 when culled, depth code q, key or EMPTY)."""
    p = _pts(points)
    va = _ViewArgs(view)
    n = p.shape[0]
    pixel = np.empty(n, np.int64)
    q = np.empty(n, np.uint64)
    key = np.empty(n, np.uint64)
    if _load().oracle_project(p.ctypes.data, n, va.M.ctypes.data, *va.args, pixel.ctypes.data, q.ctypes.data,
                              key.ctypes.data) != 0:
        raise ValueError("invalid view")
    return pixel, q, key


def clear(pixels: int) -> np.ndarray:
    fb = np.empty(pixels, np.uint64)
    _load().oracle_clear(fb.ctypes.data, pixels)
    return fb


def render_atomicmin(points, view, fb: np.ndarray | None = None) -> np.ndarray:
    """Framebuffer of per-pixel minimum keys (H*W u64, row 0 = bottom). Accumulates into `fb` if given."""
    p = _pts(points)
    va = _ViewArgs(view)
    if fb is None:
        fb = clear(va.W * va.H)
    if _load().oracle_render_atomicmin(p.ctypes.data, p.shape[0], va.M.ctypes.data, *va.args, fb.ctypes.data) != 0:
        raise ValueError("invalid view")
    return fb


def hq_accumulate(points, view, fb: np.ndarray, eps_num: int = 1, eps_den: int = 100, acc=None):
    """Second HQ pass: per-pixel (sum_r, sum_g, sum_b, count) as u64 arrays, plus an overflow flag
    (some pixel's count above 2^24)."""
    p = _pts(points)
    va = _ViewArgs(view)
    npx = va.W * va.H
    if acc is None:
        acc = tuple(np.zeros(npx, np.uint64) for _ in range(4))
    rc = _load().oracle_hq_accumulate(p.ctypes.data, p.shape[0], va.M.ctypes.data, *va.args, fb.ctypes.data,
                                      eps_num, eps_den, *(a.ctypes.data for a in acc))
    if rc == 1:
        raise ValueError("invalid view or epsilon")
    return acc, rc == 2


def resolve_basic(fb: np.ndarray, background: int = 0) -> np.ndarray:
    out = np.empty(fb.shape[0], np.uint32)
    _load().oracle_resolve_basic(fb.ctypes.data, fb.shape[0], background, out.ctypes.data)
    return out


def resolve_hq(acc, background: int = 0) -> np.ndarray:
    sr, sg, sb, cnt = acc
    out = np.empty(cnt.shape[0], np.uint32)
    _load().oracle_resolve_hq(sr.ctypes.data, sg.ctypes.data, sb.ctypes.data, cnt.ctypes.data, cnt.shape[0],
                              background, out.ctypes.data)
    return out


def bruteforce_pixel(points, view, px: int, py: int) -> int:
    """Smallest key among the points whose fragment lands on (px, py), by scanning all points."""
    p = _pts(points)
    va = _ViewArgs(view)
    return int(_load().oracle_bruteforce_pixel(p.ctypes.data, p.shape[0], va.M.ctypes.data, *va.args, px, py))
