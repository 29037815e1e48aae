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
    _fields_ = [("merge_same_pixel", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("staging", ctypes.c_int32),
                ("band_filter", ctypes.c_int32), ("band_eps_num", ctypes.c_uint32), ("band_eps_den", ctypes.c_uint32),
                ("band_bounds", ctypes.c_int32)]


class pcr_batch_tuning(ctypes.Structure):
    _fields_ = [("route", ctypes.c_int32), ("slice_words", ctypes.c_int32), ("points_per_thread", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("merge_width", ctypes.c_int32)]


class pcr_server_config(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int32), ("max_batch_views", ctypes.c_int32),
                ("framebuffer_budget_bytes", ctypes.c_uint64), ("max_frame_point_views", ctypes.c_uint64)]


class pcr_request(ctypes.Structure):
    _fields_ = [("cloud", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("hq", ctypes.c_int32), ("eps_num", ctypes.c_uint32), ("eps_den", ctypes.c_uint32),
                ("background_rgba", ctypes.c_uint32), ("reserved", ctypes.c_int32), ("view", pcr_view),
                ("d_out", ctypes.c_void_p)]


class pcr_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("batch_views", ctypes.c_int32),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double), ("done_s", ctypes.c_double)]


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
        "pcr_project_points": ([_P, ctypes.c_uint64, ctypes.POINTER(pcr_view), ctypes.c_int32, ctypes.c_int32, _P, _P,
                                _P], S),
        "pcr_render_hq_splat": ([_P, _P, ctypes.c_uint64, ctypes.POINTER(pcr_view), ctypes.c_uint32, ctypes.c_uint32,
                                 _P], S),
        "pcr_hq_accumulate": ([_P, _P, ctypes.c_uint64, ctypes.POINTER(pcr_view), ctypes.c_uint32, ctypes.c_uint32,
                               _P], S),
        "pcr_resolve": ([_P, _P, ctypes.c_uint32, ctypes.c_int32, _P], S),
        "pcr_resolve_basic": ([_P, _P, ctypes.c_uint32, ctypes.c_int32, _P], S),
        "pcr_resolve_both": ([_P, _P, _P, ctypes.c_uint32, ctypes.c_int32, _P], S),
        "pcr_framebuffer_keys": ([_P, ctypes.POINTER(_P), ctypes.POINTER(_P)], S),
        "pcr_get_device_status": ([_P, _P], S),
        "pcr_check_bounded_wait": ([_P, ctypes.c_uint32, _P], S),
        "pcr_render_frame_host": ([_P, _P, ctypes.c_uint64, ctypes.POINTER(pcr_view), ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint32, _P, _P, _P, _P, _P], S),
        "pcr_status_string": ([S], ctypes.c_char_p),
        "pcr_last_error_message": ([], ctypes.c_char_p),
        "pcr_kernel_launch_count": ([], ctypes.c_uint64),
        "pcr_cloud_create": ([_P, ctypes.c_uint64, _P, ctypes.POINTER(_P)], S),
        "pcr_cloud_destroy": ([_P], S),
        "pcr_batch_create": ([_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32,
                              ctypes.c_uint32, ctypes.c_int32, ctypes.POINTER(_P)], S),
        "pcr_batch_set_views": ([_P, _P], S),
        "pcr_batch_render": ([_P, _P], S),
        "pcr_batch_capture": ([_P, _P], S),
        "pcr_batch_launch": ([_P, _P], S),
        "pcr_batch_visible_chunks": ([_P, _P], S),
        "pcr_batch_set_tuning": ([_P, ctypes.POINTER(pcr_batch_tuning)], S),
        "pcr_batch_get_tuning": ([_P, ctypes.POINTER(pcr_batch_tuning)], S),
        "pcr_batch_autotune": ([_P, _P, ctypes.c_int32, ctypes.POINTER(pcr_batch_tuning)], S),
        "pcr_batch_destroy": ([_P], S),
        "pcr_render_views_noalloc": ([_P, ctypes.c_uint64, _P, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32, _P], S),
        "pcr_server_create": ([ctypes.POINTER(pcr_server_config), ctypes.POINTER(_P)], S),
        "pcr_server_add_cloud": ([_P, _P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32)], S),
        "pcr_server_submit": ([_P, ctypes.POINTER(pcr_request), ctypes.POINTER(ctypes.c_uint64)], S),
        "pcr_server_submit_many": ([_P, _P, ctypes.c_int32, _P], S),
        "pcr_server_poll": ([_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32], S),
        "pcr_server_destroy": ([_P], S),
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


def _tuning_dict(t: pcr_tuning) -> dict:
    return {"merge_same_pixel": t.merge_same_pixel, "blocks_per_sm": t.blocks_per_sm, "staging": t.staging,
            "band_filter": t.band_filter, "band_eps": (t.band_eps_num, t.band_eps_den), "band_bounds": t.band_bounds}


def pcr_set_tuning(fb: Framebuffer, merge_same_pixel: int | None = 0, blocks_per_sm: int = 8, staging: int = 0,
                   band_filter: int = 0, band_eps=(1, 100), band_bounds: int = 0):
    """merge_same_pixel=None restores the library defaults."""
    if merge_same_pixel is None:
        _check(load().pcr_set_tuning(fb.handle, None))
    else:
        t = pcr_tuning(int(merge_same_pixel), int(blocks_per_sm), int(staging), int(band_filter), int(band_eps[0]),
                       int(band_eps[1]), int(band_bounds))
        _check(load().pcr_set_tuning(fb.handle, ctypes.byref(t)))


def pcr_get_tuning(fb: Framebuffer):
    t = pcr_tuning()
    _check(load().pcr_get_tuning(fb.handle, ctypes.byref(t)))
    return _tuning_dict(t)


def pcr_autotune(fb: Framebuffer, points, view, stream=None):
    """Times the candidate tunings on one frame of these points and keeps the fastest; returns it."""
    ptr, n = _points_ptr(points)
    v = make_view(view)
    t = pcr_tuning()
    _check(load().pcr_autotune(fb.handle, ptr, n, ctypes.byref(v), _stream(stream), ctypes.byref(t)))
    return _tuning_dict(t)


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


def pcr_project_points(points, view, pixel=None, key=None, stream=None):
    """Per point, the fragment the view gives it: (pixel, key) as CUDA tensors, int32[n] (row * width +
    column, -1 when culled) and int64[n] (bit patterns of the u64 keys, -1 when culled). The view's width and
    height set the image. pixel and key may be given (CUDA, contiguous, n elements of 4 and 8 bytes)."""
    import torch
    ptr, n = _points_ptr(points)
    v = make_view(view)
    dev = points.device
    if pixel is None:
        pixel = torch.empty(n, dtype=torch.int32, device=dev)
    if key is None:
        key = torch.empty(n, dtype=torch.int64, device=dev)
    for t, size in ((pixel, 4), (key, 8)):
        if not t.is_cuda or t.element_size() != size or not t.is_contiguous() or t.numel() != n:
            raise ValueError("pixel and key must be contiguous CUDA tensors of n 4-byte and n 8-byte words")
    _check(load().pcr_project_points(ptr, n, ctypes.byref(v), int(view.width), int(view.height),
                                     ctypes.c_void_p(pixel.data_ptr()), ctypes.c_void_p(key.data_ptr()),
                                     _stream(stream)))
    return pixel, key


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


def pcr_resolve_both(fb: Framebuffer, out_basic, out_hq, background_rgba: int = 0, clear_after: bool = True,
                     stream=None):
    _check(load().pcr_resolve_both(fb.handle, _image_ptr(fb, out_basic), _image_ptr(fb, out_hq),
                                   background_rgba & 0xFFFFFFFF, int(clear_after), _stream(stream)))
    return out_basic, out_hq


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


def pcr_render_frame_host(fb: Framebuffer, h_points, view, d_points, d_images, h_basic, h_hq=None,
                          eps_num: int = 1, eps_den: int = 100, background_rgba: int = 0, stream=None):
    """One frame from host memory: h_points (CPU int32 (n, 4) tensor, pinned for overlap) is copied into
    d_points (CUDA tensor of the same shape), rendered, resolved, and the images land in h_basic / h_hq (CPU
    int32 tensors of W*H). d_images: CUDA int32 scratch of 2*W*H. Asynchronous on `stream`."""
    n = h_points.shape[0]
    if tuple(d_points.shape) != tuple(h_points.shape) or not d_points.is_cuda or h_points.is_cuda:
        raise ValueError("h_points must be a host tensor and d_points a CUDA tensor of the same shape")
    npx = fb.width * fb.height
    if d_images.numel() < 2 * npx or h_basic.numel() < npx or (h_hq is not None and h_hq.numel() < npx):
        raise ValueError("image buffers too small")
    v = make_view(view)
    _check(load().pcr_render_frame_host(fb.handle, ctypes.c_void_p(h_points.data_ptr()), n, ctypes.byref(v), eps_num,
                                        eps_den, background_rgba & 0xFFFFFFFF, ctypes.c_void_p(d_points.data_ptr()),
                                        ctypes.c_void_p(d_images.data_ptr()), ctypes.c_void_p(h_basic.data_ptr()),
                                        ctypes.c_void_p(h_hq.data_ptr()) if h_hq is not None else None,
                                        _stream(stream)))


def pcr_check_bounded_wait(fb: Framebuffer, rounds: int = 1024, stream=None):
    """Runs the passes' bounded barrier wait on a barrier nothing completes: sets fb's timeout bit."""
    _check(load().pcr_check_bounded_wait(fb.handle, rounds, _stream(stream)))


def pcr_status_string(status: int) -> str:
    return load().pcr_status_string(status).decode()


def pcr_last_error_message() -> str:
    return load().pcr_last_error_message().decode()


def pcr_kernel_launch_count() -> int:
    return int(load().pcr_kernel_launch_count())


def keys_to_numpy(t) -> np.ndarray:
    """int64 CUDA tensor of key bit patterns -> host uint64 array."""
    return t.cpu().numpy().view(np.uint64)


# ------------------------------------------------------------------------------------- batched rendering

class Cloud:
    """A resident cloud (pcr_cloud): keeps a reference to the points tensor, which must not change."""

    def __init__(self, handle: int, points):
        self.handle = ctypes.c_void_p(handle)
        self.points = points

    def close(self):
        if self.handle is not None and self.handle.value:
            load().pcr_cloud_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcr_cloud_create(points, stream=None) -> Cloud:
    ptr, n = _points_ptr(points)
    out = ctypes.c_void_p()
    _check(load().pcr_cloud_create(ptr, n, _stream(stream), ctypes.byref(out)))
    return Cloud(out.value, points)


class Batch:
    """A batch frame (pcr_batch) of len(fbs) views; keeps its cloud, framebuffers and outputs alive."""

    def __init__(self, handle: int, cloud: Cloud, fbs, outs):
        self.handle = ctypes.c_void_p(handle)
        self.cloud, self.fbs, self.outs = cloud, list(fbs), list(outs)

    def close(self):
        if self.handle is not None and self.handle.value:
            load().pcr_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcr_batch_create(cloud: Cloud, fbs, outs, hq: bool = False, eps_num: int = 1, eps_den: int = 100,
                     background_rgba: int = 0, clear_after: bool = True) -> Batch:
    n = len(fbs)
    if len(outs) != n:
        raise ValueError("one output per framebuffer")
    fb_arr = (ctypes.c_void_p * n)(*[fb.handle.value for fb in fbs])
    out_arr = (ctypes.c_void_p * n)(*[_image_ptr(fb, o).value for fb, o in zip(fbs, outs)])
    h = ctypes.c_void_p()
    _check(load().pcr_batch_create(cloud.handle, fb_arr, out_arr, n, int(bool(hq)), eps_num, eps_den,
                                   background_rgba & 0xFFFFFFFF, int(bool(clear_after)), ctypes.byref(h)))
    return Batch(h.value, cloud, fbs, outs)


def pcr_batch_set_views(batch: Batch, views):
    arr = (pcr_view * len(views))(*[make_view(v) for v in views])
    _check(load().pcr_batch_set_views(batch.handle, arr))


def pcr_batch_render(batch: Batch, stream=None):
    _check(load().pcr_batch_render(batch.handle, _stream(stream)))


def pcr_batch_capture(batch: Batch, stream):
    _check(load().pcr_batch_capture(batch.handle, _stream(stream)))


def pcr_batch_launch(batch: Batch, stream=None):
    _check(load().pcr_batch_launch(batch.handle, _stream(stream)))


def pcr_batch_visible_chunks(batch: Batch) -> list[int]:
    arr = (ctypes.c_uint32 * len(batch.fbs))()
    _check(load().pcr_batch_visible_chunks(batch.handle, arr))
    return list(arr)


BATCH_TUNING_FIELDS = ("route", "slice_words", "points_per_thread", "blocks_per_sm", "merge_width")


def pcr_batch_set_tuning(batch: Batch, tuning: dict | None = None):
    """tuning: a dict with the pcr_batch_tuning fields (missing ones take the defaults); None restores them."""
    if tuning is None:
        _check(load().pcr_batch_set_tuning(batch.handle, None))
        return
    d = {"route": 0, "slice_words": 1, "points_per_thread": 1, "blocks_per_sm": 4, "merge_width": 0, **tuning}
    t = pcr_batch_tuning(*[int(d[k]) for k in BATCH_TUNING_FIELDS])
    _check(load().pcr_batch_set_tuning(batch.handle, ctypes.byref(t)))


def pcr_batch_get_tuning(batch: Batch) -> dict:
    t = pcr_batch_tuning()
    _check(load().pcr_batch_get_tuning(batch.handle, ctypes.byref(t)))
    return {k: getattr(t, k) for k in BATCH_TUNING_FIELDS}


def pcr_batch_autotune(batch: Batch, stream=None, force: bool = False) -> dict:
    """Times candidate tunings on the batch's frame and keeps the fastest; returns it."""
    t = pcr_batch_tuning()
    _check(load().pcr_batch_autotune(batch.handle, _stream(stream), int(bool(force)), ctypes.byref(t)))
    return {k: getattr(t, k) for k in BATCH_TUNING_FIELDS}


def pcr_batch_destroy(batch: Batch):
    batch.close()


# ----------------------------------------------------------------------------------------------- serving

class Server:
    """A render server (pcr_server). Keeps the registered point tensors and the pending outputs alive."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)
        self.points = []
        self.outputs = {}

    def close(self):
        if self.handle is not None and self.handle.value:
            load().pcr_server_destroy(self.handle)
        self.handle = None
        self.outputs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcr_server_create(streams: int = 4, max_batch_views: int = 64, framebuffer_budget_bytes: int = 4 << 30,
                      max_frame_point_views: int = 0) -> Server:
    cfg = pcr_server_config(streams, max_batch_views, framebuffer_budget_bytes, max_frame_point_views)
    h = ctypes.c_void_p()
    _check(load().pcr_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return Server(h.value)


def pcr_server_add_cloud(server: Server, points) -> int:
    ptr, n = _points_ptr(points)
    cid = ctypes.c_int32()
    _check(load().pcr_server_add_cloud(server.handle, ptr, n, ctypes.byref(cid)))
    server.points.append(points)
    return cid.value


def _request(cloud: int, view, out, hq, eps_num, eps_den, background_rgba) -> pcr_request:
    if out.numel() != view.width * view.height or out.element_size() != 4 or not out.is_contiguous():
        raise ValueError("out must be a contiguous 4-byte tensor of width*height elements")
    return pcr_request(cloud, view.width, view.height, int(bool(hq)), eps_num, eps_den, background_rgba & 0xFFFFFFFF, 0,
                       make_view(view), out.data_ptr())


def pcr_server_submit(server: Server, cloud: int, view, out, hq: bool = False, eps_num: int = 1, eps_den: int = 100,
                      background_rgba: int = 0) -> int:
    """Queues one render of `view` (its width x height) of cloud `cloud` into the int32 CUDA tensor `out`."""
    r = _request(cloud, view, out, hq, eps_num, eps_den, background_rgba)
    rid = ctypes.c_uint64()
    _check(load().pcr_server_submit(server.handle, ctypes.byref(r), ctypes.byref(rid)))
    server.outputs[rid.value] = out
    return rid.value


def pcr_server_submit_many(server: Server, requests) -> list[int]:
    """Queues several requests at once: dicts with cloud, view, out and optional hq, eps_num, eps_den,
    background_rgba. Returns their ids."""
    arr = (pcr_request * len(requests))(*[
        _request(q["cloud"], q["view"], q["out"], q.get("hq", False), q.get("eps_num", 1), q.get("eps_den", 100),
                 q.get("background_rgba", 0)) for q in requests])
    ids = (ctypes.c_uint64 * len(requests))()
    _check(load().pcr_server_submit_many(server.handle, arr, len(requests), ids))
    for rid, q in zip(ids, requests):
        server.outputs[rid] = q["out"]
    return list(ids)


def pcr_server_poll(server: Server, max_items: int = 256, wait_ms: int = 0) -> list[dict]:
    """Completed requests, oldest first: dicts with id, status, batch_views, submit_s, start_s, done_s."""
    arr = (pcr_completion * max_items)()
    n = ctypes.c_int32()
    _check(load().pcr_server_poll(server.handle, arr, max_items, ctypes.byref(n), wait_ms))
    res = []
    for c in arr[:n.value]:
        server.outputs.pop(c.id, None)
        res.append(dict(id=c.id, status=c.status, batch_views=c.batch_views, submit_s=c.submit_s,
                        start_s=c.start_s, done_s=c.done_s))
    return res


def pcr_server_destroy(server: Server):
    server.close()


# ---------------------------------------------------------------------------------------- no allocation

PCR_NOALLOC_MAX_VIEWS = 8
PCR_NOALLOC_MAX_POINTS = 1 << 27


def pcr_render_views_noalloc(points, fbs, outs, views, hq: bool = False, eps_num: int = 1, eps_den: int = 100,
                             background_rgba: int = 0, clear_after: bool = True, stream=None):
    """One batched frame whose workspace is libpcr's fixed device array: allocates no device memory.
    Calls that overlap on the GPU race on that array (use one stream)."""
    n = len(fbs)
    if len(outs) != n or len(views) != n:
        raise ValueError("one output and one view per framebuffer")
    ptr, count = _points_ptr(points)
    fb_arr = (ctypes.c_void_p * n)(*[fb.handle.value for fb in fbs])
    out_arr = (ctypes.c_void_p * n)(*[_image_ptr(fb, o).value for fb, o in zip(fbs, outs)])
    view_arr = (pcr_view * n)(*[make_view(v) for v in views])
    _check(load().pcr_render_views_noalloc(ptr, count, fb_arr, out_arr, view_arr, n, int(bool(hq)), eps_num, eps_den,
                                           background_rgba & 0xFFFFFFFF, int(bool(clear_after)), _stream(stream)))
