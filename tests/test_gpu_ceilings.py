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


def test_fma_probe_counts_and_rates(gpu, ceil):
    """The FMA probe reports the fmas it enqueued (grid x threads x 16 chains x iters) and runs them: the
    kernel time grows with iters, and the FP32 pipes outrun the FP64 pipe."""
    import torch
    vp = ctypes.c_void_p
    ceil.pcr_ceiling_fma.argtypes = [ctypes.c_int32, ctypes.c_uint32, vp, ctypes.POINTER(ctypes.c_uint64), vp]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sink = torch.zeros(sms * 8 * 256, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    fmas = ctypes.c_uint64()
    assert ceil.pcr_ceiling_fma(2, 10, vp(sink.data_ptr()), ctypes.byref(fmas), vp(s.cuda_stream)) != 0
    assert ceil.pcr_ceiling_fma(1, 0, vp(sink.data_ptr()), ctypes.byref(fmas), vp(s.cuda_stream)) != 0

    def rate(fp64, iters):
        best = 1e30
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            assert ceil.pcr_ceiling_fma(fp64, iters, vp(sink.data_ptr()), ctypes.byref(fmas), vp(s.cuda_stream)) == 0
            b.record(s)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        assert fmas.value == sms * 8 * 256 * 16 * iters
        return fmas.value / (best * 1e-3), best

    r64, t_short = rate(1, 500)
    r64b, t_long = rate(1, 2000)
    r32, _ = rate(0, 50000)
    assert t_long > 2.5 * t_short
    assert r32 > 4 * r64b > 0
    assert int(sink.sum().item()) == 0
