"""GPU vs oracle parity through the C ABI (bit-exact keys, exact HQ sums, resolved RGB).

Tolerances: keys and HQ sums/counts are integers and must match exactly; resolved RGBA is integer
arithmetic on those sums and must match exactly as well (the +-1 LSB allowance for HQ colours is not
needed because both sides divide the same integers with the same rounding).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import scenes
from tests.helpers import RawView, axis_view, pack, rgba

pytestmark = pytest.mark.gpu

TRANSFORMS = [0, 1]  # PCR_TRANSFORM_EXACT, PCR_TRANSFORM_FP64 (both must equal the FP64 definition)


def _dev(points):
    import torch
    return torch.from_numpy(np.ascontiguousarray(points).view(np.int32)).cuda()


def _with_transform(view, transform):
    v = RawView(np.asarray(view.view_proj), view.near, view.far, view.width, view.height,
                getattr(view, "depth_mode", 0), getattr(view, "metric_scale", 1000.0), getattr(view, "ranges", None),
                transform)
    return v


def _render_basic(pcr, pts_dev, view):
    fb = pcr.pcr_create_framebuffer(view.width, view.height)
    pcr.pcr_render_atomicmin(fb, pts_dev, view)
    keys, _ = pcr.pcr_framebuffer_keys(fb)
    out = pcr.keys_to_numpy(keys)
    return fb, out


def _compare_basic(pcr, points, view, transform):
    v = _with_transform(view, transform)
    fb, got = _render_basic(pcr, _dev(points), v)
    ref = oracle.render_atomicmin(points, view)
    mism = np.flatnonzero(got != ref)
    assert mism.size == 0, f"{mism.size} pixels differ, first {mism[:5]}: got {got[mism[:3]]} want {ref[mism[:3]]}"
    import torch
    img = torch.empty(view.width * view.height, dtype=torch.int32, device="cuda")
    pcr.pcr_resolve(fb, img, background_rgba=0x00203040)
    assert np.array_equal(img.cpu().numpy().view(np.uint32), oracle.resolve_basic(ref, 0x00203040))
    return ref


@pytest.mark.parametrize("transform", TRANSFORMS)
def test_cube_1m_640x480(gpu, transform):
    """1M uniform unit-cube points, 640x480, fov 60, near 0.1, far 10, linear 40-bit depth."""
    pts = scenes.cube(1_000_000, 1)
    ref = _compare_basic(gpu, pts, scenes.cube_1m_view(), transform)
    assert np.count_nonzero(ref != oracle.EMPTY) > 20000


@pytest.mark.parametrize("transform", TRANSFORMS)
def test_lidar_ragged_1080p_basic_and_hq(gpu, transform):
    """LIDAR scene, 3M + 7 points (ragged tail), 1920x1080, basic and HQ (eps = 1 %)."""
    import torch
    pts = scenes.lidar(3_000_007, 2)
    view = scenes.lidar_1km_view()
    v = _with_transform(view, transform)
    dev = _dev(pts)
    fb = gpu.pcr_create_framebuffer(view.width, view.height, gpu.PCR_FB_HQ)
    gpu.pcr_render_hq_splat(fb, dev, v, 1, 100)
    keys, acc = gpu.pcr_framebuffer_keys(fb)
    got_keys = gpu.keys_to_numpy(keys)
    got_acc = acc.cpu().numpy().view(np.uint64)
    ref = oracle.render_atomicmin(pts, view)
    assert np.array_equal(got_keys, ref), np.count_nonzero(got_keys != ref)
    (sr, sg, sb, cnt), ovf = oracle.hq_accumulate(pts, view, ref, 1, 100)
    assert not ovf
    assert np.array_equal(got_acc[:, 0] & 0xFFFFFFFF, sr)
    assert np.array_equal(got_acc[:, 0] >> 32, sg)
    assert np.array_equal(got_acc[:, 1] & 0xFFFFFFFF, sb)
    assert np.array_equal(got_acc[:, 1] >> 32, cnt)
    img = torch.empty(view.pixels if hasattr(view, "pixels") else view.width * view.height, dtype=torch.int32,
                      device="cuda")
    gpu.pcr_resolve_basic(fb, img, 0)
    assert np.array_equal(img.cpu().numpy().view(np.uint32), oracle.resolve_basic(ref))
    gpu.pcr_resolve(fb, img, 0x01020304, clear_after=True)
    assert np.array_equal(img.cpu().numpy().view(np.uint32), oracle.resolve_hq((sr, sg, sb, cnt), 0x01020304))
    assert gpu.pcr_get_device_status(fb) == gpu.PCR_OK
    # clear_after left an empty framebuffer
    keys, acc = gpu.pcr_framebuffer_keys(fb)
    assert bool((keys == -1).all()) and bool((acc == 0).all())


@pytest.mark.parametrize("transform", TRANSFORMS)
def test_hand_built_edges(gpu, transform):
    """Frustum edges, clip planes, NaN/Inf, ties and identical points (the oracle pins' scenes)."""
    c = rgba(1, 2, 3)
    view = axis_view(64, 48, near=0.5, far=8.5)
    pts = pack([[-2.0, -2.0, -2.0], [2.0, 0.0, -2.0], [0.0, 2.0, -2.0], [0.0, 0.0, -0.5], [0.0, 0.0, -8.5],
                [0.0, 0.0, 1.0], [float("nan"), 0.0, -1.0], [float("inf"), 0.0, -1.0], [0.0, 0.0, float("-inf")],
                [0.5, 0.5, -1.0], [0.5, 0.5, -1.0], [0.5, 0.5, -1.0]],
               [c] * 9 + [rgba(0, 0, 1), rgba(255, 0, 0), rgba(0, 0, 1)])
    _compare_basic(gpu, pts, view, transform)


@pytest.mark.parametrize("transform", TRANSFORMS)
@pytest.mark.parametrize("n", [0, 1, 31, 33, 257, 4099])
def test_small_and_ragged_counts(gpu, transform, n):
    pts = scenes.cube(n, 100 + n) if n else np.zeros((0, 4), np.uint32)
    view = scenes.View.lookat((0.2, 0.1, 1.6), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 70.0, 33, 17, 0.1, 10.0)
    _compare_basic(gpu, pts, view, transform)


@pytest.mark.parametrize("transform", TRANSFORMS)
def test_metric_and_piecewise_modes(gpu, transform):
    pts = scenes.lidar(500_000, 4)
    base = scenes.lidar_1km_view(640, 360)
    mview = RawView(base.view_proj, base.near, base.far, 640, 360, depth_mode=1, metric_scale=1000.0)
    _compare_basic(gpu, pts, mview, transform)
    pview = RawView(base.view_proj, base.near, base.far, 640, 360, depth_mode=2,
                    ranges=np.array([[0.0, 10.0, 1e9], [10.0, 1e4, 1e6], [1e4, 1e7, 1e3]]))
    _compare_basic(gpu, pts, pview, transform)


@pytest.mark.parametrize("transform", TRANSFORMS)
def test_maximum_dimensions(gpu, transform):
    pts = scenes.cube(20000, 7)
    for w, h in ((16384, 1), (1, 16384), (4096, 3)):
        view = scenes.View.lookat((0.0, 0.0, 2.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, w, h, 0.1, 10.0)
        _compare_basic(gpu, pts, view, transform)


def test_order_invariance(gpu):
    pts = scenes.lidar(2_000_000, 6)
    view = scenes.lidar_1km_view()
    _, a = _render_basic(gpu, _dev(pts), view)
    sh = scenes.shuffle(pts.copy(), 3)
    _, b = _render_basic(gpu, _dev(sh), view)
    assert np.array_equal(a, b)


def test_accumulate_clear_and_errors(gpu):
    import torch
    pts = scenes.cube(100_000, 9)
    view = scenes.cube_1m_view()
    dev = _dev(pts)
    fb = gpu.pcr_create_framebuffer(view.width, view.height)
    gpu.pcr_render_atomicmin(fb, dev[:50_000], view)
    gpu.pcr_render_atomicmin(fb, dev[50_000:], view)
    keys, _ = gpu.pcr_framebuffer_keys(fb)
    assert np.array_equal(gpu.keys_to_numpy(keys), oracle.render_atomicmin(pts, view))
    gpu.pcr_clear(fb)
    torch.cuda.synchronize()
    assert bool((keys == -1).all())
    with pytest.raises(gpu.PcrError):
        gpu.pcr_render_atomicmin(fb, dev[1:].view(-1)[1:4 * 1000 + 1].view(1000, 4), view)  # misaligned
    with pytest.raises(gpu.PcrError):
        gpu.pcr_render_hq_splat(fb, dev, view)          # framebuffer without PCR_FB_HQ
    bad = RawView(view.view_proj, 1.0, 0.5, view.width, view.height)
    with pytest.raises(gpu.PcrError):
        gpu.pcr_render_atomicmin(fb, dev, bad)


def test_hq_overflow_reported(gpu):
    """More than 2^24 contributing fragments in one pixel: the HQ resolve reports PCR_ERR_OVERFLOW."""
    import torch
    n = (1 << 24) + 5
    view = axis_view(4, 4, near=0.5, far=8.5)
    one = pack([[0.0, 0.0, -1.0]], [rgba(255, 255, 255)])
    dev = _dev(one).expand(n, 4).contiguous()
    fb = gpu.pcr_create_framebuffer(4, 4, gpu.PCR_FB_HQ)
    gpu.pcr_render_hq_splat(fb, dev, view)
    img = torch.empty(16, dtype=torch.int32, device="cuda")
    gpu.pcr_resolve(fb, img)
    assert gpu.pcr_get_device_status(fb) == gpu.PCR_ERR_OVERFLOW
    assert gpu.pcr_get_device_status(fb) == gpu.PCR_OK     # status was reset


def _near_boundary_points(view, n_candidates, seed):
    """Points inside the view whose depth value t, pixel coordinate fx or clip x lies very close to a
    decision boundary of the definition (an integer code, a pixel edge, a float rounding midpoint), found
    by evaluating the transform in numpy FP64 (without fma; within ~1e-12 relative of the definition)."""
    rng = np.random.default_rng(seed)
    M = np.asarray(view.view_proj, dtype=np.float64)
    # random points in front of the camera: sample ndc and depth, map back through the inverse matrix
    inv = np.linalg.inv(M)
    ndc = rng.uniform(-1.0, 1.0, (n_candidates, 2))
    w = view.near + (min(view.far, 2000.0) - view.near) * rng.uniform(0.0, 1.0, n_candidates) ** 2
    # clip z of an OpenGL perspective matrix at depth w: (f + n) / (f - n) * w + 2 f n / (n - f)
    f_, n_ = view.far, view.near
    zc = (f_ + n_) / (f_ - n_) * w + 2.0 * f_ * n_ / (n_ - f_)
    clip = np.stack([ndc[:, 0] * w, ndc[:, 1] * w, zc, w], 1)
    world = clip @ inv.T
    world = world[:, :3] / world[:, 3:4]
    xyz = world.astype(np.float32)
    P = np.concatenate([xyz.astype(np.float64), np.ones((n_candidates, 1))], 1)
    cx, cy, ww = P @ M[0], P @ M[1], P @ M[3]
    s = 2.0 ** 40 / (view.far - view.near)
    t = (ww - view.near) * s
    ft = t - np.floor(t)
    fx = (cx.astype(np.float32) / ww.astype(np.float32) * 0.5 + 0.5) * view.width
    ffx = fx - np.floor(fx)
    c32 = cx.astype(np.float32).astype(np.float64)
    ulp = np.abs(np.spacing(cx.astype(np.float32))).astype(np.float64)
    mid = np.abs(np.abs(cx - c32) - ulp / 2) / np.maximum(ulp, 1e-300)
    sel = (np.minimum(ft, 1 - ft) < 2e-3) | (np.minimum(ffx, 1 - ffx) < 1e-4) | (mid < 1e-4)
    cols = rng.integers(0, 1 << 32, n_candidates, dtype=np.uint64).astype(np.uint32)
    return pack(xyz[sel], cols[sel]), int(sel.sum())


@pytest.mark.parametrize("transform", TRANSFORMS)
def test_adversarial_near_boundaries(gpu, transform):
    """Points selected to sit next to code, pixel-edge and float-rounding boundaries: rendered alone
    (no occlusion to hide a wrong candidate) and mixed into a scene."""
    view = scenes.lidar_1km_view(640, 360)
    pts, n_sel = _near_boundary_points(view, 3_000_000, 5)
    assert n_sel > 5000
    _compare_basic(gpu, pts, view, transform)
    mixed = np.concatenate([scenes.lidar(500_000, 8), pts])
    _compare_basic(gpu, mixed, view, transform)


@pytest.mark.parametrize("seed", range(12))
def test_random_views(gpu, seed):
    """Random cameras (eye, target, fov, near/far ratio from 20 to 1e7, resolution, depth mode) on the
    LIDAR scene and a large cube: the certified transform must equal the definition bit for bit."""
    rng = np.random.default_rng(1000 + seed)
    big = seed % 2 == 0
    pts = scenes.lidar(300_000, 30 + seed) if big else scenes.cube(300_000, 30 + seed, half=0.5 * 10.0 ** rng.uniform(-2, 3))
    centre = np.array([500.0, 500.0, 0.0]) if big else np.zeros(3)
    scale = 700.0 if big else float(np.abs(pts[:, :3].view(np.float32)).max()) * 3
    eye = centre + rng.normal(0, 1, 3) * scale
    target = centre + rng.normal(0, 0.2, 3) * scale
    d = float(np.linalg.norm(eye - centre)) + scale
    near = d * 10.0 ** rng.uniform(-5, -1)
    far = d * 10.0 ** rng.uniform(0.3, 2)
    w, h = int(rng.integers(16, 2000)), int(rng.integers(16, 1200))
    view = scenes.View.lookat(eye, target, (0.0, 0.0, 1.0) if big else (0.0, 1.0, 0.0), float(rng.uniform(20, 110)),
                              w, h, near, far)
    if seed % 3 == 1:
        view.depth_mode, view.metric_scale = 1, float(10.0 ** rng.uniform(0, 6))
    _compare_basic(gpu, pts, view, 0)


def test_certified_classification_rates(gpu):
    """Most points are decided in single precision; report the shares (for the design notes)."""
    import torch
    pts = scenes.lidar(3_000_000, 2)
    view = scenes.lidar_1km_view()
    fb = gpu.pcr_create_framebuffer(view.width, view.height)
    counts = torch.zeros(4, dtype=torch.int64, device="cuda")
    gpu.pcr_render_atomicmin_stats(fb, _dev(pts), view, counts)
    tier1, amb, fp64, tier2 = (int(c) for c in counts.cpu())
    keys, _ = gpu.pcr_framebuffer_keys(fb)
    assert np.array_equal(gpu.keys_to_numpy(keys), oracle.render_atomicmin(pts, view))
    print(f"\ncertified: tier-1 exact {tier1}, code undecided {amb}, FP64 arbiter {fp64}, tier 2 {tier2} "
          f"of {len(pts)}")
    assert tier1 > 0.9 * len(pts) * 0.8
    assert fp64 < 0.002 * len(pts) and tier2 < 0.05 * len(pts)


def test_points_around_the_camera(gpu):
    """A cloud surrounding the eye: many points lie just in front of the camera plane and far to the side, where
    the pixel error bound E is large. Tier 1 culls them when the estimate is outside the image by more than E
    (E holds at any size while it is finite); the result stays bit-exact and few points reach tier 2."""
    import torch
    rng = np.random.default_rng(5)
    n = 2_000_000
    pts = np.zeros((n, 4), np.uint32)
    pts[:, :3] = rng.uniform(-20.0, 20.0, size=(n, 3)).astype(np.float32).view(np.uint32)
    pts[:, 3] = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    view = scenes.View.lookat((0.0, 0.0, 0.0), (1.0, 0.3, 0.1), (0.0, 0.0, 1.0), 60.0, 1920, 1080, 0.01, 100.0)
    fb = gpu.pcr_create_framebuffer(view.width, view.height)
    counts = torch.zeros(4, dtype=torch.int64, device="cuda")
    gpu.pcr_render_atomicmin_stats(fb, _dev(pts), view, counts)
    tier1, amb, fp64, tier2 = (int(c) for c in counts.cpu())
    keys, _ = gpu.pcr_framebuffer_keys(fb)
    assert np.array_equal(gpu.keys_to_numpy(keys), oracle.render_atomicmin(pts, view))
    print(f"\naround the camera: tier-1 exact {tier1}, tier 2 {tier2}, FP64 arbiter {fp64} of {n}")
    assert tier2 < 0.005 * n


@pytest.mark.parametrize("merge,blocks,staging", [(0, 8, 0), (1, 8, 0), (1, 1, 0), (1, 3, 0), (0, 32, 0), (0, 8, 1),
                                                  (1, 8, 1), (1, 2, 1)])
def test_tuning_does_not_change_results(gpu, merge, blocks, staging):
    import torch
    pts = scenes.lidar(2_000_003, 12)
    view = scenes.lidar_1km_view(800, 450)
    fb = gpu.pcr_create_framebuffer(view.width, view.height, gpu.PCR_FB_HQ)
    gpu.pcr_set_tuning(fb, merge, blocks, staging)
    assert gpu.pcr_get_tuning(fb) == {"merge_same_pixel": merge, "blocks_per_sm": blocks, "staging": staging,
                                      "band_filter": 0, "band_eps": (1, 100), "band_bounds": 0}
    gpu.pcr_render_hq_splat(fb, _dev(pts), view)
    keys, acc = gpu.pcr_framebuffer_keys(fb)
    ref = oracle.render_atomicmin(pts, view)
    assert np.array_equal(gpu.keys_to_numpy(keys), ref)
    (sr, sg, sb, cnt), _ = oracle.hq_accumulate(pts, view, ref)
    a = acc.cpu().numpy().view(np.uint64)
    assert np.array_equal(a[:, 1] >> 32, cnt) and np.array_equal(a[:, 0] & 0xFFFFFFFF, sr)
    with pytest.raises(gpu.PcrError):
        gpu.pcr_set_tuning(fb, 2, 8)
    with pytest.raises(gpu.PcrError):
        gpu.pcr_set_tuning(fb, 1, 0)
    with pytest.raises(gpu.PcrError):
        gpu.pcr_set_tuning(fb, 0, 8, 2)


def test_resolve_both_equals_the_two_resolves(gpu):
    """pcr_resolve_both writes the basic and the HQ image in one pass: both equal the oracle's resolves (with a
    background), and the framebuffer is left cleared."""
    import torch
    pts = scenes.lidar(2_000_003, 31)
    view = scenes.lidar_1km_view(800, 450)
    fb = gpu.pcr_create_framebuffer(view.width, view.height, gpu.PCR_FB_HQ)
    gpu.pcr_render_hq_splat(fb, _dev(pts), view, 1, 100)
    ref = oracle.render_atomicmin(pts, view)
    sums, ovf = oracle.hq_accumulate(pts, view, ref, 1, 100)
    assert not ovf
    npx = view.width * view.height
    img_b = torch.empty(npx, dtype=torch.int32, device="cuda")
    img_h = torch.empty(npx, dtype=torch.int32, device="cuda")
    gpu.pcr_resolve_both(fb, img_b, img_h, 0x01020304, True)
    assert np.array_equal(img_b.cpu().numpy().view(np.uint32), oracle.resolve_basic(ref, 0x01020304))
    assert np.array_equal(img_h.cpu().numpy().view(np.uint32), oracle.resolve_hq(sums, 0x01020304))
    keys, acc = gpu.pcr_framebuffer_keys(fb)
    assert bool((keys == -1).all()) and bool((acc == 0).all())
    assert gpu.pcr_get_device_status(fb) == gpu.PCR_OK
    basic_only = gpu.pcr_create_framebuffer(view.width, view.height)
    with pytest.raises(gpu.PcrError):
        gpu.pcr_resolve_both(basic_only, img_b, img_h)
    basic_only.close()
    fb.close()
