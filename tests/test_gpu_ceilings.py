"""The memory-floor probes (include/pcr_ceilings.h) do the framebuffer work of the passes they stand for.

bench.py reports each pass against the time of its framebuffer operations replayed alone. That floor means
something only if the replay performs those operations: the projection must give the fragments of the FP64
definition, the pass-1 replays (one atomic per fragment, and with the stored-key read) must leave the same
minima, and the pass-2 replay the same colour sums and counts (Sections 2.1 and 2.2).
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ceil():
    from paper_1908_02681_gb300 import build as pcr_build
    lib = ctypes.CDLL(pcr_build.build_ceilings())
    vp = ctypes.c_void_p
    lib.pcr_ceiling_pattern_project.argtypes = [vp, ctypes.c_uint64, vp, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_int32, ctypes.c_int32, vp, vp, vp]
    lib.pcr_ceiling_pattern_min.argtypes = [vp, vp, ctypes.c_uint64, vp, ctypes.c_int32, vp]
    lib.pcr_ceiling_pattern_hq.argtypes = [vp, vp, ctypes.c_uint64, vp, vp, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint64, vp]
    return lib


def test_replays_do_the_passes_framebuffer_work(gpu, ceil):
    import math
    import torch
    vp = ctypes.c_void_p
    n = 1_000_003
    pts = scenes.lidar(n, 2)
    view = scenes.lidar_1km_view(640, 360)
    npx = view.width * view.height
    dev = torch.from_numpy(pts.view(np.int32)).cuda()
    pix = torch.empty(n, dtype=torch.int32, device="cuda")
    key = torch.empty(n, dtype=torch.int64, device="cuda")
    m12 = np.ascontiguousarray(np.asarray(view.view_proj, dtype=np.float64)[[0, 1, 3], :].reshape(-1))
    s = vp(torch.cuda.current_stream().cuda_stream)
    assert ceil.pcr_ceiling_pattern_project(vp(dev.data_ptr()), n, m12.ctypes.data, view.near, view.far,
                                            view.width, view.height, vp(pix.data_ptr()), vp(key.data_ptr()), s) == 0
    ref = oracle.render_atomicmin(pts, view)
    (sr, sg, sb, cnt), _ = oracle.hq_accumulate(pts, view, ref)
    for filt in (0, 1):
        keys = torch.full((npx,), -1, dtype=torch.int64, device="cuda")
        assert ceil.pcr_ceiling_pattern_min(vp(pix.data_ptr()), vp(key.data_ptr()), n, vp(keys.data_ptr()), filt,
                                            s) == 0
        got = keys.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, ref), (filt, np.count_nonzero(got != ref))
    accum = torch.zeros(2 * npx, dtype=torch.int64, device="cuda")
    nq = math.floor(view.near * (1099511627776.0 / (view.far - view.near)))
    assert ceil.pcr_ceiling_pattern_hq(vp(pix.data_ptr()), vp(key.data_ptr()), n, vp(keys.data_ptr()),
                                       vp(accum.data_ptr()), 1, 100, nq, s) == 0
    a = accum.cpu().numpy().view(np.uint64).reshape(-1, 2)
    assert np.array_equal(a[:, 0] & 0xFFFFFFFF, sr) and np.array_equal(a[:, 0] >> 32, sg)
    assert np.array_equal(a[:, 1] & 0xFFFFFFFF, sb) and np.array_equal(a[:, 1] >> 32, cnt)
    # the projection gives each point's fragment as the oracle's definition does
    o_pix, _, o_key = oracle.project(pts, view)
    assert np.array_equal(pix.cpu().numpy().astype(np.int64), o_pix)
    assert np.array_equal(key.cpu().numpy().view(np.uint64), o_key)
