"""pcr_render_frame_host: a frame from host memory (chunked upload overlapped with pass 1, pass 2,
resolves, images copied back) must give the oracle's images bit for bit, frame after frame."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu

BG = 0x00302010


@pytest.mark.parametrize("n,hq", [(9_000_011, True), (9_000_011, False), (777, True), (0, True)])
def test_frame_from_host_matches_oracle(gpu, n, hq):
    import torch
    view = scenes.lidar_1km_view(800, 450)
    npx = view.width * view.height
    fb = gpu.pcr_create_framebuffer(view.width, view.height, gpu.PCR_FB_HQ if hq else 0)
    h_img = [torch.empty(npx, dtype=torch.int32, pin_memory=True) for _ in range(2)]
    d_images = torch.empty(2 * npx, dtype=torch.int32, device="cuda")
    for seed in (51, 52):                      # two frames in a row on the same framebuffer
        pts = scenes.lidar(n, seed) if n else np.zeros((0, 4), np.uint32)
        h_pts = torch.from_numpy(pts.view(np.int32)).pin_memory() if n else torch.zeros((0, 4), dtype=torch.int32)
        d_pts = torch.empty((max(n, 1), 4), dtype=torch.int32, device="cuda")[:n]
        gpu.pcr_render_frame_host(fb, h_pts, view, d_pts, d_images, h_img[0], h_img[1] if hq else None,
                                  background_rgba=BG)
        torch.cuda.synchronize()
        ref = oracle.render_atomicmin(pts, view)
        assert np.array_equal(h_img[0].numpy().view(np.uint32), oracle.resolve_basic(ref, BG)), seed
        if hq:
            sums, _ = oracle.hq_accumulate(pts, view, ref)
            assert np.array_equal(h_img[1].numpy().view(np.uint32), oracle.resolve_hq(sums, BG)), seed
        assert gpu.pcr_get_device_status(fb) == 0
        keys, _ = gpu.pcr_framebuffer_keys(fb)
        assert bool((keys == -1).all())       # the frame left the framebuffer cleared
