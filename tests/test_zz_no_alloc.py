"""pcr_render_views_noalloc (the batched frame on libpcr's fixed device array, no allocation) against the
allocating batch entry point: two calls in a row, different views, modes and view counts, must give the
same images as pcr_batch_render (bit for bit: the batched frame is exact). Collected last, so that it also
runs after every other test in one process."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

RES = ((160, 120), (320, 180), (400, 300))
BG = 0x00203040


def _dev(points):
    import torch
    return torch.from_numpy(np.ascontiguousarray(points).view(np.int32)).cuda()


def _with_batch(gpu, dev, views, hq):
    """Images of the existing entry point (pcr_cloud_create + pcr_batch_create + pcr_batch_render)."""
    import torch
    cloud = gpu.pcr_cloud_create(dev)
    fbs = [gpu.pcr_create_framebuffer(v.width, v.height, gpu.PCR_FB_HQ if hq else 0) for v in views]
    outs = [torch.full((v.width * v.height,), -1, dtype=torch.int32, device="cuda") for v in views]
    batch = gpu.pcr_batch_create(cloud, fbs, outs, hq=hq, background_rgba=BG, clear_after=True)
    gpu.pcr_batch_set_views(batch, views)
    gpu.pcr_batch_render(batch)
    torch.cuda.synchronize()
    batch.close()
    cloud.close()
    return outs


def test_noalloc_frames_match_batch_render(gpu):
    import torch
    pts = scenes.lidar(2_000_003, 31)
    dev = _dev(pts)
    calls = [(scenes.orbit_views(6, 31, resolutions=RES), True),    # first call: 6 views, HQ
             (scenes.orbit_views(3, 32, resolutions=RES), False)]   # second call: fewer views, basic
    for views, hq in calls:
        want = _with_batch(gpu, dev, views, hq)
        fbs = [gpu.pcr_create_framebuffer(v.width, v.height, gpu.PCR_FB_HQ if hq else 0) for v in views]
        outs = [torch.full((v.width * v.height,), -1, dtype=torch.int32, device="cuda") for v in views]
        gpu.pcr_render_views_noalloc(dev, fbs, outs, views, hq=hq, background_rgba=BG)
        torch.cuda.synchronize()
        for k, (a, b) in enumerate(zip(outs, want)):
            assert bool((a == b).all()), (hq, k, int((a != b).sum()))
        for fb in fbs:
            assert gpu.pcr_get_device_status(fb) == 0


def test_noalloc_rejects_sizes_beyond_the_array(gpu):
    import torch
    lib = gpu.load()
    dev = _dev(scenes.lidar(4096, 33))
    v = scenes.orbit_views(1, 33, resolutions=((64, 48),))[0]
    fbs = [gpu.pcr_create_framebuffer(64, 48) for _ in range(gpu.PCR_NOALLOC_MAX_VIEWS + 1)]
    outs = [torch.empty(64 * 48, dtype=torch.int32, device="cuda") for _ in fbs]
    with pytest.raises(gpu.PcrError, match="views"):
        gpu.pcr_render_views_noalloc(dev, fbs, outs, [v] * len(fbs))
    # a point count above the limit is refused before anything is read
    fb_arr = (ctypes.c_void_p * 1)(fbs[0].handle.value)
    out_arr = (ctypes.c_void_p * 1)(outs[0].data_ptr())
    view_arr = (gpu.pcr_view * 1)(gpu.make_view(v))
    st = lib.pcr_render_views_noalloc(ctypes.c_void_p(dev.data_ptr()), gpu.PCR_NOALLOC_MAX_POINTS + 1, fb_arr,
                                      out_arr, view_arr, 1, 0, 1, 100, 0, 1, None)
    assert st == gpu.PCR_ERR_INVALID_ARG and "points" in gpu.pcr_last_error_message()


def test_noalloc_at_its_size_limits(gpu):
    """Exactly PCR_NOALLOC_MAX_POINTS points and PCR_NOALLOC_MAX_VIEWS views: the same images as the
    allocating batch entry point."""
    import torch
    n = gpu.PCR_NOALLOC_MAX_POINTS
    host = torch.empty((n, 4), dtype=torch.int32, pin_memory=True)
    scenes.lidar(n, 34, out=host)
    dev = host.cuda()
    views = scenes.orbit_views(gpu.PCR_NOALLOC_MAX_VIEWS, 34, resolutions=((320, 180), (256, 256)))
    want = _with_batch(gpu, dev, views, False)
    fbs = [gpu.pcr_create_framebuffer(v.width, v.height) for v in views]
    outs = [torch.full((v.width * v.height,), -1, dtype=torch.int32, device="cuda") for v in views]
    gpu.pcr_render_views_noalloc(dev, fbs, outs, views, background_rgba=BG)
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(zip(outs, want)):
        assert bool((a == b).all()), k


def test_noalloc_call_allocates_no_device_memory(gpu):
    """After a first call on the device (which looks up the array and loads the kernels), a call changes the
    device's free memory by nothing: it allocates nothing."""
    import torch
    dev = _dev(scenes.lidar(500_003, 35))
    views = scenes.orbit_views(4, 35, resolutions=RES)
    fbs = [gpu.pcr_create_framebuffer(v.width, v.height, gpu.PCR_FB_HQ) for v in views]
    outs = [torch.empty(v.width * v.height, dtype=torch.int32, device="cuda") for v in views]
    for hq in (True, False):  # warm-up: both passes' kernels loaded
        gpu.pcr_render_views_noalloc(dev, fbs, outs, views, hq=hq)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    gpu.pcr_render_views_noalloc(dev, fbs, outs, views, hq=True)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
