"""Input generators: SplitMix64 known answers, determinism, ranges and scan order (no GPU)."""
import numpy as np

import scenes


def test_splitmix64_known_answers():
    # SplitMix64 (Steele, Lea, Flood 2014) started from state 0 and from 1234567: published outputs
    assert [scenes.splitmix64_at(0, i) for i in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                              0x06C45D188009454F]
    assert [scenes.splitmix64_at(1234567, i) for i in range(2)] == [6457827717110365317, 3203168211198807973]


def test_cube_deterministic_and_in_range():
    a = scenes.cube(200000, 1, threads=1)
    b = scenes.cube(200000, 1, threads=7)
    assert np.array_equal(a, b)
    xyz = a[:, :3].view(np.float32)
    assert xyz.min() >= -0.5 and xyz.max() < 0.5
    assert np.all(a[:, 3] >> 24 == 255)
    assert not np.array_equal(a, scenes.cube(200000, 2, threads=1))


def test_lidar_deterministic_bounds_and_order():
    a = scenes.lidar(300000, 2, threads=1)
    b = scenes.lidar(300000, 2, threads=5)
    assert np.array_equal(a, b)
    xyz = a[:, :3].view(np.float32)
    assert xyz[:, 0].min() > -1.0 and xyz[:, 0].max() < 1001.0
    assert xyz[:, 1].min() > -1.0 and xyz[:, 1].max() < 1001.0
    assert xyz[:, 2].min() > -80.0 and xyz[:, 2].max() < 200.0
    # coherent order: the first 1-m strip is scanned in increasing x, the second in decreasing x
    first = xyz[:150]
    assert np.all(first[:, 1] < 1.05) and np.all(np.diff(first[:, 0]) > 0)
    second = xyz[(xyz[:, 1] > 1.05) & (xyz[:, 1] < 1.95)][:100]
    assert np.all(np.diff(second[:, 0]) < 0)


def test_shuffle_is_permutation():
    a = scenes.cube(5000, 3)
    s = scenes.shuffle(a.copy(), 4)
    assert not np.array_equal(a, s)
    key = lambda m: np.sort(m.view(np.dtype((np.void, 16))).ravel())
    assert np.array_equal(key(a), key(s))


def test_views():
    v = scenes.lidar_1km_view()
    assert v.view_proj.shape == (4, 4) and (v.width, v.height) == (1920, 1080)
    # w row is the unit forward vector: w = distance along the view axis
    f = v.view_proj[3, :3]
    assert abs(np.linalg.norm(f) - 1.0) < 1e-12
    views = scenes.orbit_views(64, 3)
    assert len(views) == 64 and [vv.width for vv in views[:3]] == [640, 1920, 3840]
