"""Pass 1's band records (pcr_tuning.band_filter; also inside pcr_render_hq_splat and pcr_render_frame_host)
and pass 2's per-pixel bounds (pcr_tuning.band_bounds). Band records:
pass 2 skips the points whose code was already beyond the HQ band of the key their pixel held in pass 1 (a
stored key only decreases, so they can never be accepted, Section 2.2). The sums and counts must equal the
oracle's exactly, in coherent and shuffled order, and a record must never serve other points, another view, a
larger eps, or a framebuffer cleared since."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu


def _dev(points):
    import torch
    return torch.from_numpy(np.ascontiguousarray(points).view(np.int32)).cuda()


def _sums(acc):
    a = acc.cpu().numpy().view(np.uint64)
    return a[:, 0] & 0xFFFFFFFF, a[:, 0] >> 32, a[:, 1] & 0xFFFFFFFF, a[:, 1] >> 32


def _expect(gpu, fb, pts, view, ref_keys, eps=(1, 100)):
    keys, acc = gpu.pcr_framebuffer_keys(fb)
    want, _ = oracle.hq_accumulate(pts, view, ref_keys, *eps)
    got = _sums(acc)
    for k in range(4):
        assert np.array_equal(got[k], want[k]), (k, int(np.count_nonzero(got[k] != want[k])))


@pytest.mark.parametrize("shuffled", [False, True])
def test_split_calls_with_band_filter(gpu, shuffled):
    pts = scenes.lidar(3_000_001, 81)
    if shuffled:
        scenes.shuffle(pts, 5)
    view = scenes.lidar_1km_view(800, 450)
    dev = _dev(pts)
    fb = gpu.pcr_create_framebuffer(view.width, view.height, gpu.PCR_FB_HQ)
    bb = int(shuffled)  # with pass 2's bounds on the shuffled cloud
    gpu.pcr_set_tuning(fb, 0, 8, 0, band_filter=1, band_eps=(1, 100), band_bounds=bb)
    assert gpu.pcr_get_tuning(fb)["band_filter"] == 1 and gpu.pcr_get_tuning(fb)["band_bounds"] == bb
    for _ in range(2):  # the second frame reuses the mask buffer
        gpu.pcr_clear(fb)
        gpu.pcr_render_atomicmin(fb, dev, view)
        gpu.pcr_hq_accumulate(fb, dev, view, 1, 100)
        ref = oracle.render_atomicmin(pts, view)
        keys, _ = gpu.pcr_framebuffer_keys(fb)
        assert np.array_equal(gpu.keys_to_numpy(keys), ref)
        _expect(gpu, fb, pts, view, ref)
        # a smaller eps may use the same record
        gpu.pcr_set_tuning(fb, 0, 8, 0, band_filter=1, band_eps=(1, 100), band_bounds=bb)
    _, acc = gpu.pcr_framebuffer_keys(fb)
    acc.zero_()
    gpu.pcr_hq_accumulate(fb, dev, view, 1, 200)
    _expect(gpu, fb, pts, view, ref, (1, 200))
    fb.close()


def test_hq_splat_and_records_not_reused(gpu):
    import torch
    a = scenes.lidar(2_000_003, 82)
    b = scenes.lidar(2_000_003, 83)
    view = scenes.lidar_1km_view(640, 360)
    da, db = _dev(a), _dev(b)
    fb = gpu.pcr_create_framebuffer(view.width, view.height, gpu.PCR_FB_HQ)
    gpu.pcr_set_tuning(fb, 0, 8, 0, band_filter=1, band_eps=(1, 100), band_bounds=1)
    gpu.pcr_render_hq_splat(fb, da, view, 1, 100)  # pass 1 records, pass 2 uses the record
    ref_a = oracle.render_atomicmin(a, view)
    _expect(gpu, fb, a, view, ref_a)
    _, acc = gpu.pcr_framebuffer_keys(fb)
    # other points against the same minima: the record of a does not apply to b
    acc.zero_()
    gpu.pcr_hq_accumulate(fb, db, view, 1, 100)
    _expect(gpu, fb, b, view, ref_a)
    # a larger eps than the record's: not used
    acc.zero_()
    gpu.pcr_hq_accumulate(fb, da, view, 1, 20)
    _expect(gpu, fb, a, view, ref_a, (1, 20))
    # another view (same points): not used
    other = scenes.lidar_1km_view(640, 360)
    other.view_proj = np.array(other.view_proj, copy=True)
    other.view_proj[0, 3] += 1e-3
    acc.zero_()
    gpu.pcr_hq_accumulate(fb, da, other, 1, 100)
    _expect(gpu, fb, a, other, ref_a)
    # cleared: the record is dropped; pass 1 of b without recording, then pass 2 of a (with a's pointer)
    gpu.pcr_clear(fb)
    gpu.pcr_set_tuning(fb, 0, 8, 0, band_filter=0)
    gpu.pcr_render_atomicmin(fb, db, view)
    gpu.pcr_hq_accumulate(fb, da, view, 1, 100)
    ref_b = oracle.render_atomicmin(b, view)
    _expect(gpu, fb, a, view, ref_b)
    fb.close()


def test_frame_from_host_buffers_with_records(gpu):
    """pcr_render_frame_host records in chunks (tile-aligned) and its pass 2 uses the record: both images equal
    the oracle's at a size that takes 8 chunks."""
    import torch
    n = 9_000_017
    host = torch.empty((n, 4), dtype=torch.int32, pin_memory=True)
    scenes.lidar(n, 84, out=host)
    pts = host.numpy().view(np.uint32)
    view = scenes.lidar_1km_view(960, 540)
    fb = gpu.pcr_create_framebuffer(view.width, view.height, gpu.PCR_FB_HQ)
    gpu.pcr_set_tuning(fb, 0, 8, 0, band_filter=1, band_eps=(1, 100), band_bounds=1)
    npx = view.width * view.height
    d_pts = torch.empty_like(host, device="cuda")
    d_img = torch.empty(2 * npx, dtype=torch.int32, device="cuda")
    h_basic = torch.empty(npx, dtype=torch.int32, pin_memory=True)
    h_hq = torch.empty(npx, dtype=torch.int32, pin_memory=True)
    gpu.pcr_render_frame_host(fb, host, view, d_pts, d_img, h_basic, h_hq, 1, 100)
    torch.cuda.synchronize()
    ref = oracle.render_atomicmin(pts, view)
    sums, _ = oracle.hq_accumulate(pts, view, ref)
    assert np.array_equal(h_basic.numpy().view(np.uint32), oracle.resolve_basic(ref))
    assert np.array_equal(h_hq.numpy().view(np.uint32), oracle.resolve_hq(sums))
    fb.close()


@pytest.mark.parametrize("bounds", [0, 1])
@pytest.mark.parametrize("eps", [(1, 100), (3, 7), (1, 1 << 20), (5, 3), ((1 << 24) - 2, 2), ((1 << 24) - 1, 2)])
def test_band_bounds_and_their_limit(gpu, eps, bounds):
    """With band_bounds, pass 2 tests decided codes against per-pixel bounds {qmin, qmin + floor(eps_num (qmin +
    Nq) / eps_den)} while eps_num (2^40 + Nq) + eps_den 2^40 <= 2^64, and against the stored key beyond (METRIC
    view, Nq = 0: (2^24 - 2) / 2 is the last eps inside, (2^24 - 1) / 2 the first outside; the others take the
    invariant-divisor division at several divisors). Points of another cloud against the minima: where the
    minimum is the empty code, the u64 test of the largest eps accepts every point (its left side wraps), the
    bounds would not; the sums must equal the oracle's in every case."""
    from tests.helpers import RawView
    a = scenes.lidar(1_000_003, 85)
    b = scenes.lidar(1_000_003, 86)
    base = scenes.lidar_1km_view(640, 360)
    view = RawView(base.view_proj, base.near, base.far, 640, 360, depth_mode=1, metric_scale=1000.0)
    fb = gpu.pcr_create_framebuffer(view.width, view.height, gpu.PCR_FB_HQ)
    gpu.pcr_set_tuning(fb, 0, 8, 0, band_bounds=bounds)
    gpu.pcr_render_atomicmin(fb, _dev(a), view)
    ref = oracle.render_atomicmin(a, view)
    for pts in (a, b):
        _, acc = gpu.pcr_framebuffer_keys(fb)
        acc.zero_()
        gpu.pcr_hq_accumulate(fb, _dev(pts), view, *eps)
        _expect(gpu, fb, pts, view, ref, eps)
    fb.close()


@pytest.mark.parametrize("n", [0, 1, 31, 63, 64, 65, 129, 4099])
def test_small_counts_with_both_options(gpu, n):
    """Band records and band bounds on counts below, at and just past one 64-point tile (the records' unit):
    keys, sums and counts equal the oracle's, and an empty cloud records nothing and adds nothing."""
    import torch
    pts = scenes.cube(n, 300 + n) if n else np.zeros((0, 4), np.uint32)
    view = scenes.View.lookat((0.2, 0.1, 1.6), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 70.0, 33, 17, 0.1, 10.0)
    fb = gpu.pcr_create_framebuffer(view.width, view.height, gpu.PCR_FB_HQ)
    gpu.pcr_set_tuning(fb, 0, 8, 0, band_filter=1, band_eps=(1, 100), band_bounds=1)
    dev = _dev(pts) if n else torch.zeros((0, 4), dtype=torch.int32, device="cuda")
    for _ in range(2):
        gpu.pcr_clear(fb)
        gpu.pcr_render_hq_splat(fb, dev, view, 1, 100)
        ref = oracle.render_atomicmin(pts, view)
        keys, _ = gpu.pcr_framebuffer_keys(fb)
        assert np.array_equal(gpu.keys_to_numpy(keys), ref)
        _expect(gpu, fb, pts, view, ref)
    assert gpu.pcr_get_device_status(fb) == gpu.PCR_OK
    fb.close()


@pytest.mark.parametrize("metric", [False, True])
@pytest.mark.parametrize("eps", [(1, 100), (3, 7), (1, 1 << 20), (5, 3), (1 << 23, 3)])
def test_band_records_across_eps(gpu, eps, metric):
    """Band records written and used at several eps (the record's high-word test with its integer and fraction
    parts of eps, and its constant C from Nq), on a LINEAR (Nq > 0) and a METRIC (Nq = 0) view, shuffled so that
    the records drop many points: sums and counts equal the oracle's."""
    from tests.helpers import RawView
    pts = scenes.lidar(1_500_007, 87)
    scenes.shuffle(pts, 9)
    base = scenes.lidar_1km_view(640, 360)
    view = RawView(base.view_proj, base.near, base.far, 640, 360, depth_mode=1 if metric else 0,
                   metric_scale=1000.0)
    dev = _dev(pts)
    fb = gpu.pcr_create_framebuffer(view.width, view.height, gpu.PCR_FB_HQ)
    gpu.pcr_set_tuning(fb, 0, 8, 0, band_filter=1, band_eps=eps)
    gpu.pcr_render_hq_splat(fb, dev, view, *eps)
    ref = oracle.render_atomicmin(pts, view)
    keys, _ = gpu.pcr_framebuffer_keys(fb)
    assert np.array_equal(gpu.keys_to_numpy(keys), ref)
    _expect(gpu, fb, pts, view, ref, eps)
    fb.close()
