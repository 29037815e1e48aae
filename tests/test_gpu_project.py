"""Per-point parity (pcr_project_points): every point's pixel and key against the FP64 definition of the oracle.

The framebuffer tests compare what each pixel keeps, so a point that loses its pixel is never looked at. Here
every point's own fragment is compared, element by element: the decisions of the single-precision tiers are
checked for all points, including those placed behind others and those next to pixel, depth-code and clip
boundaries (Sections 1 and 2.1).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import scenes
from tests.helpers import axis_view, pack, rgba
from tests.test_gpu_parity import _near_boundary_points

pytestmark = pytest.mark.gpu


def _dev(points):
    import torch
    return torch.from_numpy(np.ascontiguousarray(points).view(np.int32)).cuda()


def _project(gpu, pts, view, transform):
    view.transform = transform
    pix, key = gpu.pcr_project_points(_dev(pts), view)
    return pix.cpu().numpy().astype(np.int64), key.cpu().numpy().view(np.uint64)


def _check(gpu, pts, view, transforms=(0, 1)):
    o_pix, _, o_key = oracle.project(pts, view)
    for t in transforms:
        pix, key = _project(gpu, pts, view, t)
        bad = np.flatnonzero((pix != o_pix) | (key != o_key))
        assert bad.size == 0, (t, bad.size, bad[:5], pix[bad[:5]], o_pix[bad[:5]], key[bad[:5]], o_key[bad[:5]])
    return o_pix


def test_cube_and_lidar(gpu):
    o = _check(gpu, scenes.cube(1_000_003, 1), scenes.cube_1m_view())
    assert np.count_nonzero(o >= 0) > 900_000
    o = _check(gpu, scenes.lidar(3_000_001, 2), scenes.lidar_1km_view(800, 450))
    assert np.count_nonzero(o >= 0) > 2_000_000


def test_points_near_every_boundary(gpu):
    """Points next to pixel edges, depth-code integers and the clip planes, where the tiers hand over."""
    view = scenes.lidar_1km_view(640, 360)
    pts, n_sel = _near_boundary_points(view, 3_000_000, 5)
    assert n_sel > 5000
    _check(gpu, pts, view)


@pytest.mark.parametrize("seed", range(8))
def test_random_views(gpu, seed):
    rng = np.random.default_rng(2000 + seed)
    big = seed % 2 == 0
    pts = scenes.lidar(300_000, 50 + seed) if big else scenes.cube(300_000, 50 + seed, half=0.5 * 10.0 ** rng.uniform(-2, 3))
    centre = np.array([500.0, 500.0, 0.0]) if big else np.zeros(3)
    scale = 700.0 if big else float(np.abs(pts[:, :3].view(np.float32)).max()) * 3
    eye = centre + rng.normal(0, 1, 3) * scale
    target = centre + rng.normal(0, 0.2, 3) * scale
    d = float(np.linalg.norm(eye - centre)) + scale
    view = scenes.View.lookat(eye, target, (0.0, 0.0, 1.0) if big else (0.0, 1.0, 0.0), float(rng.uniform(20, 110)),
                              int(rng.integers(16, 2000)), int(rng.integers(16, 1200)), d * 10.0 ** rng.uniform(-5, -1),
                              d * 10.0 ** rng.uniform(0.3, 2))
    if seed % 3 == 1:
        view.depth_mode, view.metric_scale = 1, float(10.0 ** rng.uniform(0, 6))
    _check(gpu, pts, view)


def test_points_around_the_camera(gpu):
    """Points just in front of the camera and far to the side: large pixel bounds, culled in tier 1."""
    rng = np.random.default_rng(5)
    n = 1_000_000
    xyz = rng.uniform(-20.0, 20.0, size=(n, 3)).astype(np.float32)
    pts = pack(xyz, rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32))
    view = scenes.View.lookat((0.0, 0.0, 0.0), (1.0, 0.3, 0.1), (0.0, 0.0, 1.0), 60.0, 1920, 1080, 0.01, 100.0)
    _check(gpu, pts, view)


def test_city_sample(gpu):
    """20M points of the city scene (near 1 cm, far 10 km, coordinates up to 5 km) at 3840x2160."""
    pts = scenes.lidar(20_000_000, 4, scenes.lidar_params_city())
    _check(gpu, pts, scenes.city_view(4))


def test_piecewise_depth_and_special_values(gpu):
    """Piecewise depth with one, two and three ranges (the exact transform selects each range's constants by a
    branch on w), and NaN / infinity / huge coordinates: z = -inf gives w = +inf on this camera, which must not
    select a range the view does not have."""
    rng = np.random.default_rng(9)
    xyz = np.column_stack([rng.uniform(-6, 6, 20000), rng.uniform(-6, 6, 20000), rng.uniform(-9, 0, 20000)])
    pts = pack(xyz, np.full(20000, rgba(1, 2, 3)))
    special = pack([[np.nan, 0, -1], [np.inf, 0, -1], [0, -np.inf, -1], [1e38, 1e38, -1e38], [0, 0, -0.5],
                    [0, 0, -8.5], [-1, -1, -1], [0.999, 0.999, -1], [0, 0, -np.inf], [0, 0, -3.4e38],
                    [0.5, 0.5, -3.4e38]], np.full(11, rgba(9, 8, 7)))
    for ranges in ([[0.5, 8.5, 1e6]],
                   [[0.5, 1.0, 1e9], [1.0, 8.5, 1e6]],
                   [[0.5, 1.0, 1e9], [1.0, 4.0, 1e6], [4.0, 8.5, 1e5]]):
        v = axis_view(depth_mode=2)
        v.ranges = np.array(ranges)
        _check(gpu, pts, v, transforms=(0, 1, 2))
        _check(gpu, special, v)
    _check(gpu, special, axis_view())


def test_double_float_mismatch_is_rare(gpu):
    view = scenes.lidar_1km_view(800, 450)
    pts = scenes.lidar(2_000_000, 6)
    o_pix, _, o_key = oracle.project(pts, view)
    pix, key = _project(gpu, pts, view, 2)
    assert np.mean(pix != o_pix) < 1e-3 and np.mean(key != o_key) < 1e-2


def test_arguments(gpu):
    import torch
    view = scenes.cube_1m_view()
    pts = _dev(scenes.cube(100, 1))
    with pytest.raises(ValueError):
        gpu.pcr_project_points(pts, view, pixel=torch.empty(99, dtype=torch.int32, device="cuda"))
    pix, key = gpu.pcr_project_points(pts[:0], view)
    assert pix.numel() == 0 and key.numel() == 0
