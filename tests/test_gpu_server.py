"""Serving (pcr_server): requests over several resident clouds, mixed resolutions and modes, merged into shared
frames on several streams. Every image must equal the same request rendered alone (through the server and
through the single-view entry points) bit for bit, and a sample of them the oracle's image."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu

RES = ((160, 120), (320, 180), (256, 256), (400, 300))
BG = 0x00445566


def _dev(points):
    import torch
    return torch.from_numpy(np.ascontiguousarray(points).view(np.int32)).cuda()


def _drain(gpu, server, n, timeout_s=60.0):
    import time
    got, t0 = [], time.time()
    while len(got) < n:
        got += gpu.pcr_server_poll(server, 256, 100)
        assert time.time() - t0 < timeout_s, f"{len(got)} of {n} requests completed"
    return got


def _single(gpu, dev, view, hq):
    """The request rendered through the single-view entry points (Section 2.1 / 2.2 passes, then resolve)."""
    import torch
    fb = gpu.pcr_create_framebuffer(view.width, view.height, gpu.PCR_FB_HQ if hq else 0)
    out = torch.empty(view.width * view.height, dtype=torch.int32, device="cuda")
    if hq:
        gpu.pcr_render_hq_splat(fb, dev, view, 1, 100)
        gpu.pcr_resolve(fb, out, BG)
    else:
        gpu.pcr_render_atomicmin(fb, dev, view)
        gpu.pcr_resolve_basic(fb, out, BG)
    torch.cuda.synchronize()
    return out


def test_served_images_equal_alone_and_oracle(gpu):
    import torch
    clouds = [scenes.lidar(1_500_001, 21), scenes.lidar(700_000, 22)]
    devs = [_dev(p) for p in clouds]
    torch.cuda.synchronize()
    server = gpu.pcr_server_create(streams=3, max_batch_views=8, framebuffer_budget_bytes=256 << 20)
    ids = [gpu.pcr_server_add_cloud(server, d) for d in devs]
    views = scenes.orbit_views(30, 41, resolutions=RES)
    reqs = []
    for i, v in enumerate(views):
        c, hq = i % 2 if i % 5 else 1, (i % 3 == 0)
        out = torch.full((v.width * v.height,), -1, dtype=torch.int32, device="cuda")
        reqs.append([None, c, v, hq, out])
    # the first 20 at once (they share frames by group), the rest one by one
    first = gpu.pcr_server_submit_many(server, [dict(cloud=ids[c], view=v, out=o, hq=hq, background_rgba=BG)
                                                for _, c, v, hq, o in reqs[:20]])
    for q, rid in zip(reqs, first):
        q[0] = rid
    for q in reqs[20:]:
        q[0] = gpu.pcr_server_submit(server, ids[q[1]], q[2], q[4], hq=q[3], background_rgba=BG)
    done = {d["id"]: d for d in _drain(gpu, server, len(reqs))}
    assert all(d["status"] == 0 for d in done.values())
    assert max(done[rid]["batch_views"] for rid in first) > 1    # requests of one group shared a frame
    groups = {}
    for rid, c, v, hq, o in reqs[:20]:
        groups.setdefault((c, hq), []).append(done[rid]["batch_views"])
    assert all(max(b) > 1 for b in groups.values() if len(b) > 1)
    for d in done.values():
        assert d["submit_s"] <= d["start_s"] <= d["done_s"]
    # alone: each request through the same server, one at a time, and through the single-view entry points
    for k, (rid, c, v, hq, out) in enumerate(reqs):
        alone = torch.full_like(out, -1)
        gpu.pcr_server_submit(server, ids[c], v, alone, hq=hq, background_rgba=BG)
        (d,) = _drain(gpu, server, 1)
        assert d["status"] == 0 and d["batch_views"] == 1
        assert bool((alone == out).all()), k
        assert bool((_single(gpu, devs[c], v, hq) == out).all()), k
        if k % 7 == 0:
            ref = oracle.render_atomicmin(clouds[c], v)
            if hq:
                sums, _ = oracle.hq_accumulate(clouds[c], v, ref)
                want = oracle.resolve_hq(sums, BG)
            else:
                want = oracle.resolve_basic(ref, BG)
            assert np.array_equal(out.cpu().numpy().view(np.uint32), want), k
    gpu.pcr_server_destroy(server)


def test_small_budget_and_rejections(gpu):
    import torch
    pts = scenes.lidar(400_000, 23)
    dev = _dev(pts)
    torch.cuda.synchronize()
    big = scenes.orbit_views(1, 5, resolutions=((400, 300),))[0]
    budget = 400 * 300 * 24 + 256                                  # exactly one HQ 400x300 framebuffer
    server = gpu.pcr_server_create(streams=2, max_batch_views=4, framebuffer_budget_bytes=budget)
    cid = gpu.pcr_server_add_cloud(server, dev)
    views = scenes.orbit_views(6, 9, resolutions=((400, 300), (160, 120)))
    outs = []
    for v in views:
        outs.append(torch.empty(v.width * v.height, dtype=torch.int32, device="cuda"))
        gpu.pcr_server_submit(server, cid, v, outs[-1], hq=True, background_rgba=BG)
    done = _drain(gpu, server, len(views))
    assert all(d["status"] == 0 for d in done)
    for v, o in zip(views, outs):
        assert bool((_single(gpu, dev, v, True) == o).all())
    huge = scenes.orbit_views(1, 5, resolutions=((800, 600),))[0]
    o = torch.empty(800 * 600, dtype=torch.int32, device="cuda")
    with pytest.raises(gpu.PcrError):
        gpu.pcr_server_submit(server, cid, huge, o, hq=True)        # larger than the whole budget
    with pytest.raises(gpu.PcrError):
        gpu.pcr_server_submit(server, 7, big, outs[0])               # unknown cloud
    from tests.helpers import RawView
    fp64 = RawView(big.view_proj, big.near, big.far, big.width, big.height, transform=1)
    with pytest.raises(gpu.PcrError):
        gpu.pcr_server_submit(server, cid, fp64, outs[0])            # served views use the EXACT transform
    gpu.pcr_server_destroy(server)


def test_frame_work_cap(gpu):
    """max_frame_point_views: with a cap of 2.5 clouds' worth, no frame holds more than 2 requests, and a
    cap below one request still runs each request (alone); the images do not change."""
    import torch
    pts = scenes.lidar(1_000_000, 24)
    dev = _dev(pts)
    torch.cuda.synchronize()
    views = scenes.orbit_views(7, 25, resolutions=((320, 180), (160, 120)))
    for cap, most in ((2_500_000, 2), (1000, 1)):
        server = gpu.pcr_server_create(streams=1, max_batch_views=8, framebuffer_budget_bytes=256 << 20,
                                       max_frame_point_views=cap)
        cid = gpu.pcr_server_add_cloud(server, dev)
        outs = [torch.empty(v.width * v.height, dtype=torch.int32, device="cuda") for v in views]
        gpu.pcr_server_submit_many(server, [dict(cloud=cid, view=v, out=o, background_rgba=BG)
                                            for v, o in zip(views, outs)])
        done = _drain(gpu, server, len(views))
        assert all(d["status"] == 0 for d in done)
        assert max(d["batch_views"] for d in done) == most
        for v, o in zip(views, outs):
            assert bool((_single(gpu, dev, v, False) == o).all())
        gpu.pcr_server_destroy(server)

