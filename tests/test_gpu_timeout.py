"""Failure detection without a GPU fault: the point passes' bounded barrier wait, run on a barrier that
nothing completes, gives up, sets the framebuffer's timeout bit (read as PCR_ERR_TIMEOUT) and leaves the
context and the framebuffer usable."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_framebuffer_stays_usable(gpu):
    import torch
    view = scenes.cube_1m_view()
    fb = gpu.pcr_create_framebuffer(view.width, view.height)
    per_round = []
    for rounds in (1024, 16384):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        gpu.pcr_check_bounded_wait(fb, rounds)
        b.record()
        b.synchronize()
        per_round.append(a.elapsed_time(b) * 1e3 / rounds)
        assert gpu.pcr_get_device_status(fb) == gpu.PCR_ERR_TIMEOUT
        assert gpu.pcr_get_device_status(fb) == gpu.PCR_OK      # the status was reset
    print(f"\nbounded wait: {per_round[-1]:.3f} us per round; the passes' limit of 2^18 rounds "
          f"~ {per_round[-1] * (1 << 18) / 1e6:.2f} s")
    # the context and the framebuffer still work
    pts = scenes.cube(200_003, 7)
    gpu.pcr_render_atomicmin(fb, torch.from_numpy(pts.view(np.int32)).cuda(), view)
    keys, _ = gpu.pcr_framebuffer_keys(fb)
    assert np.array_equal(gpu.keys_to_numpy(keys), oracle.render_atomicmin(pts, view))
    assert gpu.pcr_get_device_status(fb) == gpu.PCR_OK
    with pytest.raises(gpu.PcrError):
        gpu.pcr_check_bounded_wait(fb, (1 << 18) + 1)
