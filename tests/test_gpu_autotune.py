"""The autotuners (pcr_autotune for single views, pcr_batch_autotune for batched frames) and every tuning they
can pick: a tuning changes how the work is launched, never the result. Every tuned frame must equal the oracle
bit for bit (Sections 2.1 and 2.2), the autotuners must return a tuning from their candidate sets and keep it,
the batch autotuner's cache must round-trip through its file, and on the batched workload (64 orbit views of a
20M-point cloud at mixed resolutions) the tuned frame must not be slower than the default one."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu

RES = ((160, 120), (320, 180), (400, 300))
BG = 0x00112233


def _dev(points):
    import torch
    return torch.from_numpy(np.ascontiguousarray(points).view(np.int32)).cuda()


@pytest.fixture(scope="module")
def scene():
    """2M LIDAR points, 6 orbit views, and the oracle's images of both modes for each view."""
    pts = scenes.lidar(2_000_003, 41)
    views = scenes.orbit_views(6, 41, resolutions=RES)
    want = {}
    for i, v in enumerate(views):
        ref = oracle.render_atomicmin(pts, v)
        sums, _ = oracle.hq_accumulate(pts, v, ref)
        want[(i, False)] = oracle.resolve_basic(ref, BG)
        want[(i, True)] = oracle.resolve_hq(sums, BG)
    return pts, views, want


def _batch(gpu, dev, views, hq):
    import torch
    cloud = gpu.pcr_cloud_create(dev)
    fbs = [gpu.pcr_create_framebuffer(v.width, v.height, gpu.PCR_FB_HQ if hq else 0) for v in views]
    outs = [torch.full((v.width * v.height,), -1, dtype=torch.int32, device="cuda") for v in views]
    batch = gpu.pcr_batch_create(cloud, fbs, outs, hq=hq, background_rgba=BG, clear_after=True)
    gpu.pcr_batch_set_views(batch, views)
    return batch, outs


def _images_equal(outs, want, hq):
    import torch
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        got = o.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want[(i, hq)]), (i, hq, int(np.count_nonzero(got != want[(i, hq)])))


TUNINGS = [
    dict(route=1),
    dict(route=2),
    dict(route=1, slice_words=2, points_per_thread=2),
    dict(route=1, slice_words=4, blocks_per_sm=2),
    dict(route=1, merge_width=8),
    dict(route=1, merge_width=16, points_per_thread=2),
    dict(route=1, merge_width=32, slice_words=4, blocks_per_sm=3),
]


@pytest.mark.parametrize("hq", [False, True])
def test_every_batch_tuning_gives_the_oracle_images(gpu, scene, hq):
    pts, views, want = scene
    dev = _dev(pts)
    batch, outs = _batch(gpu, dev, views, hq)
    for t in TUNINGS:
        gpu.pcr_batch_set_tuning(batch, t)
        got = gpu.pcr_batch_get_tuning(batch)
        assert all(got[k] == v for k, v in t.items()), (t, got)
        for o in outs:
            o.fill_(-1)
        gpu.pcr_batch_render(batch)
        _images_equal(outs, want, hq)
    for bad in (dict(route=3), dict(slice_words=3), dict(points_per_thread=4), dict(blocks_per_sm=0),
                dict(merge_width=4)):
        with pytest.raises(gpu.PcrError):
            gpu.pcr_batch_set_tuning(batch, bad)
    gpu.pcr_batch_set_tuning(batch, None)
    assert gpu.pcr_batch_get_tuning(batch) == dict(route=0, slice_words=1, points_per_thread=1, blocks_per_sm=4,
                                                   merge_width=0)
    batch.close()


def test_captured_frame_follows_tuning_and_views(gpu, scene):
    """A captured frame is re-captured at launch when its tuning changes, and (for single-view passes, whose view
    constants live in the graph) when its views change."""
    import torch
    pts, views, want = scene
    dev = _dev(pts)
    batch, outs = _batch(gpu, dev, views, True)
    s = torch.cuda.Stream()
    gpu.pcr_batch_set_tuning(batch, dict(route=2))
    gpu.pcr_batch_capture(batch, s)
    gpu.pcr_batch_launch(batch, s)
    s.synchronize()
    _images_equal(outs, want, True)
    # new views on the captured single-view frame: the next launch re-captures
    other = scenes.orbit_views(6, 42, resolutions=RES)
    gpu.pcr_batch_set_views(batch, other)
    gpu.pcr_batch_launch(batch, s)
    s.synchronize()
    for i, (v, o) in enumerate(zip(other, outs)):
        ref = oracle.render_atomicmin(pts, v)
        sums, _ = oracle.hq_accumulate(pts, v, ref)
        assert np.array_equal(o.cpu().numpy().view(np.uint32), oracle.resolve_hq(sums, BG)), i
    # back to the first views with the batch kernel: tuning change, then views change (no re-capture needed)
    gpu.pcr_batch_set_tuning(batch, dict(route=1, slice_words=2, merge_width=16))
    gpu.pcr_batch_set_views(batch, views)
    gpu.pcr_batch_launch(batch, s)
    s.synchronize()
    _images_equal(outs, want, True)
    batch.close()


def test_batch_autotune_picks_keeps_and_caches(gpu, scene, tmp_path, monkeypatch):
    pts, views, want = scene
    dev = _dev(pts)
    cache = tmp_path / "autotune.tsv"
    monkeypatch.setenv("PCR_AUTOTUNE_CACHE", str(cache))
    batch, outs = _batch(gpu, dev, views, True)
    best = gpu.pcr_batch_autotune(batch, force=True)
    assert best["route"] in (1, 2) and best["slice_words"] in (1, 2, 4) and best["points_per_thread"] in (1, 2)
    assert best["blocks_per_sm"] in (2, 3, 4) and best["merge_width"] in (0, 8, 16, 32)
    assert gpu.pcr_batch_get_tuning(batch) == best
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].split("\t")[1] == "hq"
    assert lines[0].split("\t")[-1] == " ".join(str(best[k]) for k in gpu.BATCH_TUNING_FIELDS)
    for o in outs:
        o.fill_(-1)
    gpu.pcr_batch_render(batch)
    _images_equal(outs, want, True)
    # a second batch of the same shape takes the remembered tuning without timing anything
    batch2, outs2 = _batch(gpu, dev, views, True)
    gpu.pcr_batch_set_tuning(batch2, dict(route=1, merge_width=8))
    assert gpu.pcr_batch_autotune(batch2, force=False) == best
    assert gpu.pcr_batch_get_tuning(batch2) == best
    assert len(cache.read_text().splitlines()) == 1
    gpu.pcr_batch_render(batch2)
    _images_equal(outs2, want, True)
    # the basic mode is another key
    batch3, outs3 = _batch(gpu, dev, views, False)
    gpu.pcr_batch_autotune(batch3)
    lines = cache.read_text().splitlines()
    assert len(lines) == 2 and lines[1].split("\t")[1] == "basic"
    gpu.pcr_batch_render(batch3)
    _images_equal(outs3, want, False)
    for b in (batch, batch2, batch3):
        b.close()


def test_autotuned_batched_workload_not_slower(gpu, tmp_path, monkeypatch):
    """The batched workload: 64 orbit views of a 20M-point cloud at 640x480 / 1920x1080 / 3840x2160, basic mode,
    replayed from a CUDA graph. The tuned frame gives the same images and is not slower than the default."""
    import torch
    monkeypatch.setenv("PCR_AUTOTUNE_CACHE", str(tmp_path / "autotune.tsv"))
    n = 20_000_000
    host = torch.empty((n, 4), dtype=torch.int32, pin_memory=True)
    scenes.lidar(n, 3, out=host)
    dev = host.cuda()
    views = scenes.orbit_views(64, 3, resolutions=((640, 480), (1920, 1080), (3840, 2160)))
    cloud = gpu.pcr_cloud_create(dev)
    fbs = [gpu.pcr_create_framebuffer(v.width, v.height) for v in views]
    outs = [torch.empty(v.width * v.height, dtype=torch.int32, device="cuda") for v in views]
    batch = gpu.pcr_batch_create(cloud, fbs, outs, clear_after=True)
    gpu.pcr_batch_set_views(batch, views)
    s = torch.cuda.Stream()

    def timed():
        gpu.pcr_batch_capture(batch, s)
        for _ in range(2):
            gpu.pcr_batch_launch(batch, s)
        best = 1e30
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            gpu.pcr_batch_launch(batch, s)
            b.record(s)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    t_default = timed()
    ref = [o.clone() for o in outs]
    tuned = gpu.pcr_batch_autotune(batch, s, force=True)
    t_tuned = timed()
    for k, (a, b) in enumerate(zip(outs, ref)):
        assert bool((a == b).all()), k
    print(f"\nbatched 64 views x 20M: default {t_default:.3f} ms, tuned {t_tuned:.3f} ms with {tuned}")
    assert t_tuned <= 1.03 * t_default, (t_tuned, t_default, tuned)
    batch.close()
    cloud.close()


def test_single_view_autotune(gpu):
    pts = scenes.lidar(3_000_001, 43)
    view = scenes.lidar_1km_view(800, 450)
    fb = gpu.pcr_create_framebuffer(view.width, view.height, gpu.PCR_FB_HQ)
    dev = _dev(pts)
    best = gpu.pcr_autotune(fb, dev, view)
    assert best["merge_same_pixel"] in (0, 1) and best["staging"] in (0, 1) and best["blocks_per_sm"] in (2, 4, 6, 8)
    assert best["band_filter"] in (0, 1) and best["band_eps"] == (1, 100) and best["band_bounds"] in (0, 1)
    assert gpu.pcr_get_tuning(fb) == best
    keys, acc = gpu.pcr_framebuffer_keys(fb)
    assert np.all(gpu.keys_to_numpy(keys) == oracle.EMPTY)  # cleared at the end
    gpu.pcr_render_hq_splat(fb, dev, view)
    ref = oracle.render_atomicmin(pts, view)
    assert np.array_equal(gpu.keys_to_numpy(keys), ref)
    (sr, sg, sb, cnt), _ = oracle.hq_accumulate(pts, view, ref)
    a = acc.cpu().numpy().view(np.uint64)
    assert np.array_equal(a[:, 1] >> 32, cnt) and np.array_equal(a[:, 0] & 0xFFFFFFFF, sr)
    fb.close()
