"""Batched rendering (pcr_cloud / pcr_batch): every view of a batch must equal the oracle bit for bit (keys,
HQ sums and counts, images), with chunk culling, one persistent launch per pass, and CUDA-graph replay."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu

RES = ((160, 120), (320, 180), (400, 300))


def _dev(points):
    import torch
    return torch.from_numpy(np.ascontiguousarray(points).view(np.int32)).cuda()


def _frame(gpu, dev, views, hq, clear_after=False):
    import torch
    cloud = gpu.pcr_cloud_create(dev)
    fbs = [gpu.pcr_create_framebuffer(v.width, v.height, gpu.PCR_FB_HQ if hq else 0) for v in views]
    outs = [torch.empty(v.width * v.height, dtype=torch.int32, device="cuda") for v in views]
    batch = gpu.pcr_batch_create(cloud, fbs, outs, hq=hq, background_rgba=0x00112233, clear_after=clear_after)
    gpu.pcr_batch_set_views(batch, views)
    return cloud, fbs, outs, batch


def _check_view(gpu, pts, view, fb, out, hq):
    keys, acc = gpu.pcr_framebuffer_keys(fb)
    got = gpu.keys_to_numpy(keys)
    ref = oracle.render_atomicmin(pts, view)
    assert np.array_equal(got, ref), np.count_nonzero(got != ref)
    if hq:
        sums, _ = oracle.hq_accumulate(pts, view, ref)
        a = acc.cpu().numpy().view(np.uint64)
        assert np.array_equal(a[:, 0] & 0xFFFFFFFF, sums[0]) and np.array_equal(a[:, 0] >> 32, sums[1])
        assert np.array_equal(a[:, 1] & 0xFFFFFFFF, sums[2]) and np.array_equal(a[:, 1] >> 32, sums[3])
        want = oracle.resolve_hq(sums, 0x00112233)
    else:
        want = oracle.resolve_basic(ref, 0x00112233)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("hq", [False, True])
def test_batch_orbit_views_match_oracle(gpu, hq):
    pts = scenes.lidar(3_000_003, 3)
    views = scenes.orbit_views(9, 3, resolutions=RES)
    dev = _dev(pts)
    cloud, fbs, outs, batch = _frame(gpu, dev, views, hq)
    gpu.pcr_batch_render(batch)
    counts = gpu.pcr_batch_visible_chunks(batch)
    n_chunks = (len(pts) + 1023) // 1024
    assert all(0 < c <= n_chunks for c in counts) and min(counts) < n_chunks
    for v, fb, out in zip(views, fbs, outs):
        _check_view(gpu, pts, v, fb, out, hq)


def test_batch_matches_single_view_launches(gpu):
    pts = scenes.lidar(2_000_000, 5)
    views = scenes.orbit_views(6, 11, resolutions=RES)
    dev = _dev(pts)
    cloud, fbs, outs, batch = _frame(gpu, dev, views, False)
    gpu.pcr_batch_render(batch)
    for v, fb in zip(views, fbs):
        single = gpu.pcr_create_framebuffer(v.width, v.height)
        gpu.pcr_render_atomicmin(single, dev, v)
        a, _ = gpu.pcr_framebuffer_keys(fb)
        b, _ = gpu.pcr_framebuffer_keys(single)
        assert bool((a == b).all())


def test_graph_replay_and_view_update(gpu):
    import torch
    pts = scenes.lidar(1_500_000, 7)
    views = scenes.orbit_views(5, 13, resolutions=RES)
    dev = _dev(pts)
    cloud, fbs, outs, batch = _frame(gpu, dev, views, True, clear_after=True)
    stream = torch.cuda.Stream()
    gpu.pcr_batch_capture(batch, stream)
    gpu.pcr_batch_launch(batch, stream)
    stream.synchronize()
    first = [o.clone() for o in outs]
    gpu.pcr_batch_launch(batch, stream)          # framebuffers were cleared by the frame: same images
    stream.synchronize()
    assert all(bool((a == b).all()) for a, b in zip(first, outs))
    for v, o in zip(views, first):
        ref = oracle.render_atomicmin(pts, v)
        sums, _ = oracle.hq_accumulate(pts, v, ref)
        assert np.array_equal(o.cpu().numpy().view(np.uint32), oracle.resolve_hq(sums, 0x00112233))
    new_views = scenes.orbit_views(5, 14, resolutions=RES)
    new_views = [scenes.View(nv.view_proj, nv.near, nv.far, v.width, v.height) for nv, v in zip(new_views, views)]
    gpu.pcr_batch_set_views(batch, new_views)
    gpu.pcr_batch_launch(batch, stream)
    stream.synchronize()
    for v, o in zip(new_views, outs):
        ref = oracle.render_atomicmin(pts, v)
        sums, _ = oracle.hq_accumulate(pts, v, ref)
        assert np.array_equal(o.cpu().numpy().view(np.uint32), oracle.resolve_hq(sums, 0x00112233))


def test_batch_edge_cases(gpu):
    import torch
    from tests.helpers import axis_view, pack, rgba
    # non-finite points (never culled chunk), a ragged last chunk, points on the frustum edges
    pts = np.concatenate([scenes.cube(5000, 2), pack([[np.nan, 0, -1], [0, 0, np.inf], [-2, -2, -2], [2, 0, -2]],
                                                     [rgba(1, 2, 3)] * 4)])
    views = [scenes.cube_1m_view(), scenes.View.lookat((0.4, 0.2, 1.8), (0, 0, 0), (0, 1, 0), 70.0, 33, 17, 0.1, 10.0),
             axis_view(64, 48, near=0.5, far=8.5)]
    dev = _dev(pts)
    cloud, fbs, outs, batch = _frame(gpu, dev, views, False)
    gpu.pcr_batch_render(batch)
    for v, fb, out in zip(views, fbs, outs):
        _check_view(gpu, pts, v, fb, out, False)
    with pytest.raises(gpu.PcrError):
        gpu.pcr_batch_create(cloud, [fbs[0], fbs[0]], [outs[0], outs[0]])
    pview = axis_view(64, 48, depth_mode=2)
    pview.ranges = [[0.0, 10.0, 1e9]]
    with pytest.raises(gpu.PcrError):
        gpu.pcr_batch_set_views(batch, [views[0], views[1], pview])


def test_batch_maximum_view_count(gpu):
    """PCR_MAX_BATCH_VIEWS (256) views in one frame, graph-captured: sampled views against the oracle; 257
    views are refused."""
    import torch
    pts = scenes.lidar(500_001, 61)
    dev = _dev(pts)
    views = scenes.orbit_views(256, 61, resolutions=((32, 24), (48, 27), (40, 40)))
    cloud, fbs, outs, batch = _frame(gpu, dev, views, False, clear_after=True)
    stream = torch.cuda.Stream()
    gpu.pcr_batch_capture(batch, stream)
    gpu.pcr_batch_launch(batch, stream)
    stream.synchronize()
    for k in (0, 1, 127, 200, 255):
        want = oracle.resolve_basic(oracle.render_atomicmin(pts, views[k]), 0x00112233)
        assert np.array_equal(outs[k].cpu().numpy().view(np.uint32), want), k
    extra = fbs + [gpu.pcr_create_framebuffer(32, 24)]
    with pytest.raises(gpu.PcrError):
        gpu.pcr_batch_create(cloud, extra, outs + [torch.empty(32 * 24, dtype=torch.int32, device="cuda")])
