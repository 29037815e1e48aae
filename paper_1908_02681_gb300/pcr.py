"""Python binding of libpcr (include/pcr.h): the same entry points, argument marshalling only.

PyTorch supplies device memory and streams: points are CUDA tensors of shape (n, 4) and 4-byte dtype
(float32 x, y, z bits + RGBA8 word), output images are CUDA int32/uint32 tensors of width * height
words, and the stream defaults to torch's current stream. Every step of the rasterizer runs in the
library's CUDA kernels; there is no CPU or PyTorch fallback, and loading fails loudly when the library
has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpcr.so")

PCR_OK, PCR_ERR_INVALID_ARG, PCR_ERR_CUDA, PCR_ERR_OOM, PCR_ERR_OVERFLOW, PCR_ERR_TIMEOUT = range(6)
PCR_DEPTH_LINEAR, PCR_DEPTH_METRIC, PCR_DEPTH_PIECEWISE = range(3)
PCR_TRANSFORM_EXACT, PCR_TRANSFORM_FP64, PCR_TRANSFORM_DOUBLE_FLOAT = range(3)
PCR_FB_HQ = 1
MAX_DEPTH_RANGES = 8
EMPTY_KEY = 0xFFFFFFFFFFFFFFFF


class PcrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} [status {status}]")
        self.status = status


class pcr_view(ctypes.Structure):
    _fields_ = [("view_proj", ctypes.c_double * 16), ("near_plane", ctypes.c_double), ("far_plane", ctypes.c_double),
                ("depth_mode", ctypes.c_int32), ("transform", ctypes.c_int32), ("metric_scale", ctypes.c_double),
                ("n_ranges", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ranges", (ctypes.c_double * 3) * MAX_DEPTH_RANGES)]


class pcr_tuning(ctypes.Structure):
    _fields_ = [("merge_same_pixel", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]


_P = ctypes.c_void_p
_lib = None


def _declare(lib):
    S = ctypes.c_int
    sig = {
        "pcr_create_framebuffer": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(_P)], S),
        "pcr_destroy_framebuffer": ([_P], S),
        "pcr_framebuffer_info": ([_P, _P, _P, _P], S),
        "pcr_set_tuning": ([_P, ctypes.POINTER(pcr_tuning)], S),
        "pcr_get_tuning": ([_P, ctypes.POINTER(pcr_tuning)], S),
        "pcr_autotune": ([_P, _P, ctypes.c_uint64, ctypes.POINTER(pcr_view), _P, ctypes.POINTER(pcr_tuning)], S),
        "pcr_clear": ([_P, _P], S),
        "pcr_render_atomicmin": ([_P, _P, ctypes.c_uint64, ctypes.POINTER(pcr_view), _P], S),
        "pcr_render_atomicmin_stats": ([_P, _P, ctypes.c_uint64, ctypes.POINTER(pcr_view), _P, _P], S),
        "pcr_render_hq_splat": ([_P, _P, ctypes.c_uint64, ctypes.POINTER(pcr_view), ctypes.c_uint32, ctypes.c_uint32,
                                 _P], S),
        "pcr_hq_accumulate": ([_P, _P, ctypes.c_uint64, ctypes.POINTER(pcr_view), ctypes.c_uint32, ctypes.c_uint32,
                               _P], S),
        "pcr_resolve": ([_P, _P, ctypes.c_uint32, ctypes.c_int32, _P], S),
        "pcr_resolve_basic": ([_P, _P, ctypes.c_uint32, ctypes.c_int32, _P], S),
        "pcr_framebuffer_keys": ([_P, ctypes.POINTER(_P), ctypes.POINTER(_P)], S),
        "pcr_get_device_status": ([_P, _P], S),
        "pcr_status_string": ([S], ctypes.c_char_p),
        "pcr_last_error_message": ([], ctypes.c_char_p),
        "pcr_kernel_launch_count": ([], ctypes.c_uint64),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def load(path: str | None = None):
    """Load libpcr.so (built in-tree by `paper_1908_02681_gb300.build`). Raises if it is missing."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libpcr.so not found at {p}: build it first (python -c 'import __graft_entry__ as g; "
                               f"g.build()')")
        _lib = _declare(ctypes.CDLL(p))
    return _lib


def _check(status: int):
    if status != PCR_OK:
        lib = load()
        raise PcrError(status, lib.pcr_last_error_message().decode() or lib.pcr_status_string(status).decode())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def make_view(view) -> pcr_view:
    """Marshal a view object (view_proj, near, far and optional depth_mode, metric_scale, ranges,
    transform attributes) into the C struct."""
    v = pcr_view()
    m = np.ascontiguousarray(np.asarray(view.view_proj, dtype=np.float64).reshape(16))
    for i in range(16):
        v.view_proj[i] = float(m[i])
    v.near_plane = float(view.near)
    v.far_plane = float(view.far)
    v.depth_mode = int(getattr(view, "depth_mode", PCR_DEPTH_LINEAR))
    v.transform = int(getattr(view, "transform", PCR_TRANSFORM_EXACT))
    v.metric_scale = float(getattr(view, "metric_scale", 1000.0))
    ranges = getattr(view, "ranges", None)
    if ranges is not None:
        r = np.asarray(ranges, dtype=np.float64).reshape(-1, 3)
        v.n_ranges = r.shape[0]
        for k in range(min(r.shape[0], MAX_DEPTH_RANGES)):
            for j in range(3):
                v.ranges[k][j] = float(r[k, j])
    return v


def _points_ptr(points):
    if not points.is_cuda:
        raise ValueError("points must be a CUDA tensor")
    if points.dim() != 2 or points.shape[1] != 4 or points.element_size() != 4 or not points.is_contiguous():
        raise ValueError("points must be a contiguous (n, 4) tensor of a 4-byte dtype")
    return ctypes.c_void_p(points.data_ptr()), points.shape[0]


class _DeviceArray:
    """Zero-copy view of library-owned device memory for torch.as_tensor (CUDA array interface)."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 2, "strides": None, "stream": None}


class Framebuffer:
    """Owns a pcr_framebuffer handle; destroyed with the object (or by close())."""

    def __init__(self, handle: int, width: int, height: int, flags: int):
        self.handle = ctypes.c_void_p(handle)
        self.width, self.height, self.flags = width, height, flags

    @property
    def pixels(self) -> int:
        return self.width * self.height

    def close(self):
        if self.handle is not None and self.handle.value:
            load().pcr_destroy_framebuffer(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcr_create_framebuffer(width: int, height: int, flags: int = 0) -> Framebuffer:
    out = ctypes.c_void_p()
    _check(load().pcr_create_framebuffer(width, height, flags, ctypes.byref(out)))
    return Framebuffer(out.value, width, height, flags)


def pcr_destroy_framebuffer(fb: Framebuffer):
    fb.close()


def pcr_framebuffer_info(fb: Framebuffer):
    w, h, f = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_uint32()
    _check(load().pcr_framebuffer_info(fb.handle, ctypes.byref(w), ctypes.byref(h), ctypes.byref(f)))
    return w.value, h.value, f.value


def pcr_set_tuning(fb: Framebuffer, merge_same_pixel: int | None = 0, blocks_per_sm: int = 8):
    """merge_same_pixel=None restores the library defaults."""
    if merge_same_pixel is None:
        _check(load().pcr_set_tuning(fb.handle, None))
    else:
        t = pcr_tuning(int(merge_same_pixel), int(blocks_per_sm))
        _check(load().pcr_set_tuning(fb.handle, ctypes.byref(t)))


def pcr_get_tuning(fb: Framebuffer):
    t = pcr_tuning()
    _check(load().pcr_get_tuning(fb.handle, ctypes.byref(t)))
    return {"merge_same_pixel": t.merge_same_pixel, "blocks_per_sm": t.blocks_per_sm}


def pcr_autotune(fb: Framebuffer, points, view, stream=None):
    """Times the candidate tunings on one frame of these points and keeps the fastest; returns it."""
    ptr, n = _points_ptr(points)
    v = make_view(view)
    t = pcr_tuning()
    _check(load().pcr_autotune(fb.handle, ptr, n, ctypes.byref(v), _stream(stream), ctypes.byref(t)))
    return {"merge_same_pixel": t.merge_same_pixel, "blocks_per_sm": t.blocks_per_sm}


def pcr_clear(fb: Framebuffer, stream=None):
    _check(load().pcr_clear(fb.handle, _stream(stream)))


def pcr_render_atomicmin(fb: Framebuffer, points, view, stream=None):
    ptr, n = _points_ptr(points)
    v = make_view(view)
    _check(load().pcr_render_atomicmin(fb.handle, ptr, n, ctypes.byref(v), _stream(stream)))


def pcr_render_atomicmin_stats(fb: Framebuffer, points, view, counts, stream=None):
    """counts: CUDA int64 tensor of >= 4 elements (accumulated, not cleared)."""
    ptr, n = _points_ptr(points)
    v = make_view(view)
    if not counts.is_cuda or counts.element_size() != 8 or counts.numel() < 4:
        raise ValueError("counts must be a CUDA tensor of at least 4 8-byte words")
    _check(load().pcr_render_atomicmin_stats(fb.handle, ptr, n, ctypes.byref(v), ctypes.c_void_p(counts.data_ptr()),
                                             _stream(stream)))


def pcr_render_hq_splat(fb: Framebuffer, points, view, eps_num: int = 1, eps_den: int = 100, stream=None):
    ptr, n = _points_ptr(points)
    v = make_view(view)
    _check(load().pcr_render_hq_splat(fb.handle, ptr, n, ctypes.byref(v), eps_num, eps_den, _stream(stream)))


def pcr_hq_accumulate(fb: Framebuffer, points, view, eps_num: int = 1, eps_den: int = 100, stream=None):
    ptr, n = _points_ptr(points)
    v = make_view(view)
    _check(load().pcr_hq_accumulate(fb.handle, ptr, n, ctypes.byref(v), eps_num, eps_den, _stream(stream)))


def _image_ptr(fb: Framebuffer, out):
    if not out.is_cuda or out.element_size() != 4 or not out.is_contiguous() or out.numel() != fb.pixels:
        raise ValueError("output must be a contiguous CUDA tensor of width * height 4-byte words")
    return ctypes.c_void_p(out.data_ptr())


def pcr_resolve(fb: Framebuffer, out, background_rgba: int = 0, clear_after: bool = False, stream=None):
    _check(load().pcr_resolve(fb.handle, _image_ptr(fb, out), background_rgba & 0xFFFFFFFF, int(clear_after),
                              _stream(stream)))
    return out


def pcr_resolve_basic(fb: Framebuffer, out, background_rgba: int = 0, clear_after: bool = False, stream=None):
    _check(load().pcr_resolve_basic(fb.handle, _image_ptr(fb, out), background_rgba & 0xFFFFFFFF, int(clear_after),
                                    _stream(stream)))
    return out


def pcr_framebuffer_keys(fb: Framebuffer):
    """(keys, accum) as zero-copy torch tensors over the library's device memory: keys int64[pixels]
    (bit patterns of the u64 keys), accum int64[pixels, 2] or None."""
    import torch
    k, a = ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().pcr_framebuffer_keys(fb.handle, ctypes.byref(k), ctypes.byref(a)))
    keys = torch.as_tensor(_DeviceArray(k.value, (fb.pixels,), "<i8", fb), device="cuda")
    acc = None if not a.value else torch.as_tensor(_DeviceArray(a.value, (fb.pixels, 2), "<i8", fb), device="cuda")
    return keys, acc


def pcr_get_device_status(fb: Framebuffer, stream=None) -> int:
    """Synchronises the stream and returns (and resets) the framebuffer's device status code."""
    return int(load().pcr_get_device_status(fb.handle, _stream(stream)))


def pcr_status_string(status: int) -> str:
    return load().pcr_status_string(status).decode()


def pcr_last_error_message() -> str:
    return load().pcr_last_error_message().decode()


def pcr_kernel_launch_count() -> int:
    return int(load().pcr_kernel_launch_count())


def keys_to_numpy(t) -> np.ndarray:
    """int64 CUDA tensor of key bit patterns -> host uint64 array."""
    return t.cpu().numpy().view(np.uint64)
