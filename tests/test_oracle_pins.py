"""Pins of the oracle against what the paper and the mathematics fix (no GPU).

Each check is a plain function so that `test_oracle_mutants.py` can run the same set against copies of
the oracle with planted mistakes and show that every such mistake fails at least one check.

What pins what:
  * exact dyadic scenes: every FP64/FP32 operation of the definition is exact, so the oracle must equal
    exact rational arithmetic (Fractions): projection rows, signs, pixel mapping and orientation,
    pixel indexing, depth quantisation, key packing (Sections 2.1).
  * general scenes: the oracle must agree with exact rational arithmetic wherever the exact value is
    farther from a decision boundary than the FP64/FP32 rounding bound of the definition.
  * hand-built scenes with known winners, tie-break by the smaller colour (Section 2.1), the empty
    sentinel, culling boundaries, the 40-bit cap, the paper's printed capacity figures (Section 2.1).
  * brute force: per-pixel minimum by scanning all points, and a numpy scatter-min of the per-point
    fragments, on random tiny scenes; shuffled order gives the same framebuffer.
  * high-quality splatting (Section 2.2): inclusive 1 % band on exact depths, colour averages with
    round-half-up, count/sentinel invariants.
"""
from __future__ import annotations

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import scenes
from tests.helpers import RawView, axis_view, pack, rgba

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TWO40 = 1 << 40


# ----------------------------------------------------------------------------- exact dyadic projection

DYADIC_M = np.array([[0.5, 0.25, -0.125, 0.75],
                     [-0.25, 0.5, 0.375, -0.5],
                     [7.0, 7.0, 7.0, 7.0],        # clip z: not used by the method
                     [0.125, -0.25, -1.0, 2.0]])


def _dyadic_points(rng, n):
    """Points whose clip w is a power of two (so every operation of the definition is exact)."""
    x = rng.integers(-256, 257, n) / 64.0
    y = rng.integers(-256, 257, n) / 64.0
    w = rng.choice([0.5, 1.0, 2.0, 4.0], n)
    z = 0.125 * x - 0.25 * y + 2.0 - w
    col = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    return pack(np.stack([x, y, z], 1), col), np.stack([x, y, z], 1), col


def _exact_fragment(M, p, col, view):
    """Exact rational evaluation of the definition (Sections 2.1): None when culled, else (pixel, q, key)."""
    P = [Fraction(float(v)) for v in p] + [Fraction(1)]
    row = lambda r: sum(Fraction(float(M[r][j])) * P[j] for j in range(4))
    cx, cy, w = row(0), row(1), row(3)
    near, far = Fraction(view.near), Fraction(view.far)
    if not (near <= w < far):
        return None
    fx = (cx / w / 2 + Fraction(1, 2)) * view.width
    fy = (cy / w / 2 + Fraction(1, 2)) * view.height
    if not (0 <= fx < view.width and 0 <= fy < view.height):
        return None
    if view.depth_mode == 0:
        t = (w - near) * Fraction(TWO40) / (far - near)
    else:
        t = w * Fraction(view.metric_scale)
    q = min(math.floor(t), TWO40 - 2)
    return math.floor(fy) * view.width + math.floor(fx), q, (q << 24) | (int(col) & 0xFFFFFF)


def check_exact_dyadic_linear():
    rng = np.random.default_rng(11)
    view = RawView(DYADIC_M, 0.5, 8.5, 64, 48)          # far - near = 8, so s = 2^37 exactly
    pts, xyz, col = _dyadic_points(rng, 3000)
    pixel, q, key = oracle.project(pts, view)
    n_vis = 0
    for i in range(len(pts)):
        ex = _exact_fragment(DYADIC_M, xyz[i], col[i], view)
        if ex is None:
            assert pixel[i] == -1, i
        else:
            n_vis += 1
            assert (pixel[i], int(q[i]), int(key[i])) == ex, (i, xyz[i])
    assert n_vis > 500


def check_exact_dyadic_metric():
    rng = np.random.default_rng(12)
    view = RawView(DYADIC_M, 0.25, 6.0, 40, 30, depth_mode=1, metric_scale=1000.0)
    pts, xyz, col = _dyadic_points(rng, 2000)
    pixel, q, key = oracle.project(pts, view)
    n_vis = 0
    for i in range(len(pts)):
        ex = _exact_fragment(DYADIC_M, xyz[i], col[i], view)
        if ex is None:
            assert pixel[i] == -1
        else:
            n_vis += 1
            assert (pixel[i], int(q[i]), int(key[i])) == ex
    assert n_vis > 300


def check_frustum_edges():
    """ndc exactly -1 maps to pixel 0 (kept); ndc exactly +1 maps to W (culled); w = near kept, w = far culled."""
    view = axis_view(64, 48, near=0.5, far=8.5)
    c = rgba(1, 2, 3)
    pts = pack([[-2.0, -2.0, -2.0],   # ndc (-1, -1): fx = fy = 0 -> pixel 0
                [2.0, 0.0, -2.0],     # ndc x = +1: fx = W -> culled
                [0.0, 2.0, -2.0],     # ndc y = +1: fy = H -> culled
                [0.0, 0.0, -0.5],     # w = near: kept
                [0.0, 0.0, -8.5],     # w = far: culled
                [0.0, 0.0, 1.0],      # behind the camera
                [float("nan"), 0.0, -1.0],
                [float("inf"), 0.0, -1.0],
                [0.0, 0.0, float("-inf")]], [c] * 9)
    pixel, q, key = oracle.project(pts, view)
    assert pixel.tolist() == [0, -1, -1, 24 * 64 + 32, -1, -1, -1, -1, -1]
    assert int(q[0]) == int((2.0 - 0.5) * (1 << 37)) and int(q[3]) == 0
    assert int(key[3]) == c & 0xFFFFFF


def check_pixel_orientation():
    """Row 0 is the bottom row; pixel index is py * W + px (non-square image)."""
    view = axis_view(8, 4, near=0.5, far=8.5)
    # w = 1: ndc = (x, y); fx = (x/2 + 1/2) * 8, fy = (y/2 + 1/2) * 4
    pts = pack([[-0.875, -0.875, -1.0],   # fx = 0.5, fy = 0.25 -> (0, 0)
                [0.875, -0.875, -1.0],    # fx = 7.5 -> (7, 0)
                [-0.875, 0.875, -1.0],    # fy = 3.75 -> (0, 3)
                [0.125, 0.375, -1.0]],    # fx = 4.5, fy = 2.75 -> (4, 2)
               [rgba(9, 9, 9)] * 4)
    pixel, _, _ = oracle.project(pts, view)
    assert pixel.tolist() == [0, 7, 3 * 8, 2 * 8 + 4]


def check_known_winners_and_tiebreak():
    view = axis_view(16, 16, near=0.5, far=8.5)
    red, blue1, green = rgba(255, 0, 0), rgba(0, 0, 1), rgba(0, 200, 0)
    pts = pack([[0.0, 0.0, -4.0], [0.0, 0.0, -2.0], [0.0, 0.0, -3.0],      # pixel A: nearest (w=2) wins
                [0.5, 0.5, -1.0], [0.5, 0.5, -1.0],                            # pixel B: equal depth
                [-0.5, -0.5, -1.0], [-0.5, -0.5, -1.0]],                       # pixel C: identical points
               [green, red, blue1, blue1, red, green, green])
    fb = oracle.render_atomicmin(pts, view)
    a = 8 * 16 + 8
    b = int((0.75 * 16)) * 16 + int(0.75 * 16)
    c = int(0.25 * 16) * 16 + int(0.25 * 16)
    q2 = int((2.0 - 0.5) * (1 << 37))
    q1 = int((1.0 - 0.5) * (1 << 37))
    assert int(fb[a]) == (q2 << 24) | (red & 0xFFFFFF)
    # equal depth: the smaller 24-bit colour value wins; byte 0 = R is least significant, so pure red
    # (0x0000FF) beats B = 1 (0x010000)
    assert int(fb[b]) == (q1 << 24) | 0x0000FF
    assert int(fb[c]) == (q1 << 24) | (green & 0xFFFFFF)
    assert int(np.count_nonzero(fb != oracle.EMPTY)) == 3


def check_empty_and_sentinel():
    view = axis_view(12, 10)
    fb = oracle.render_atomicmin(np.zeros((0, 4), np.uint32), view)
    assert fb.shape == (120,) and np.all(fb == 0xFFFFFFFFFFFFFFFF)
    img = oracle.resolve_basic(fb, background=0x11223344)
    assert np.all(img == 0x11223344)
    # points all culled -> still empty
    fb = oracle.render_atomicmin(pack([[0, 0, 5.0], [0, 0, -100.0]], [1, 2]), view)
    assert np.all(fb == oracle.EMPTY)


def check_depth_cap_and_capacity():
    """Section 2.1: 40 bits hold about one trillion values; at millimetre precision that is one
    million km. Depth codes are capped at 2^40 - 2 so that no key reaches the empty sentinel."""
    with open(os.path.join(GOLDEN, "paper_depth_capacity.json")) as f:
        g = json.load(f)
    view = axis_view(4, 4, near=0.5, far=1e10, depth_mode=1, metric_scale=g["units_per_metre"])
    w_ok = g["max_distance_m"]
    pts = pack([[0, 0, -w_ok], [0, 0, -2.0 * w_ok], [0, 0, -1.25]], [0, 0, 0])
    pixel, q, _ = oracle.project(pts, view)
    assert int(q[0]) == g["codes_at_max_distance"] and int(q[0]) < TWO40 - 2
    assert int(q[1]) == TWO40 - 2
    assert int(q[2]) == 1250
    assert (1 << g["depth_bits"]) >= g["approx_values"]


def check_paper_clear_value():
    """Section 2.1: the paper clears to 0xffffffffff000000 (maximum depth, black). Every point key has a
    depth code of at most 2^40 - 2 and therefore orders below both that value and the all-ones sentinel."""
    with open(os.path.join(GOLDEN, "paper_clear_value.json")) as f:
        g = json.load(f)
    paper_clear = int(g["clear_value"], 16)
    assert paper_clear >> 24 == (1 << 40) - 1 and paper_clear & 0xFFFFFF == g["background_rgb"]
    biggest_key = ((TWO40 - 2) << 24) | 0xFFFFFF
    assert biggest_key < paper_clear < oracle.EMPTY
    # a framebuffer cleared with the paper's value resolves to black (its colour bits), alpha 255
    img = oracle.resolve_basic(np.array([paper_clear], np.uint64))
    assert int(img[0]) == 0xFF000000


def check_bruteforce_tiny():
    rng_seeds = [1, 2, 3]
    for seed in rng_seeds:
        pts = scenes.cube(3000, seed)
        view = scenes.View.lookat((0.3, -0.2, 2.0), (0.0, 0.05, 0.0), (0.0, 1.0, 0.0), 50.0, 24, 18, 0.1, 10.0)
        fb = oracle.render_atomicmin(pts, view)
        for py in range(18):
            for px in range(24):
                assert int(fb[py * 24 + px]) == oracle.bruteforce_pixel(pts, view, px, py)
        # scatter-min of the per-point fragments (numpy) gives the same buffer
        pixel, _, key = oracle.project(pts, view)
        ref = np.full(24 * 18, oracle.EMPTY, np.uint64)
        vis = pixel >= 0
        np.minimum.at(ref, pixel[vis], key[vis])
        assert np.array_equal(ref, fb)
        assert np.count_nonzero(vis) > 1000


def check_order_invariance():
    pts = scenes.lidar(20000, 5)
    view = scenes.lidar_1km_view(64, 36)
    fb1 = oracle.render_atomicmin(pts, view)
    sh = scenes.shuffle(pts.copy(), 9)
    assert not np.array_equal(sh, pts)
    fb2 = oracle.render_atomicmin(sh, view)
    assert np.array_equal(fb1, fb2)


def _fp_bounds_check(pts, view, expect_checked):
    """Compare oracle fragments with exact rational values wherever rounding cannot matter."""
    M = np.asarray(view.view_proj, dtype=np.float64)
    pixel, q, _ = oracle.project(pts, view)
    xyz = pts[:, :3].view(np.float32)
    near, far = Fraction(view.near), Fraction(view.far)
    s_exact = Fraction(TWO40) / (far - near)
    u53 = Fraction(1, 1 << 53)
    checked = 0
    for i in range(pts.shape[0]):
        P = [Fraction(float(v)) for v in xyz[i]] + [Fraction(1)]
        rows = []
        for r in (0, 1, 3):
            terms = [Fraction(float(M[r][j])) * P[j] for j in range(4)]
            rows.append((sum(terms), sum(abs(t) for t in terms)))
        (cx, tcx), (cy, tcy), (w, tw) = rows
        ew = 3 * u53 * tw * 2                       # three fma roundings, doubled for safety
        if w - ew < near and w + ew >= near or w - ew < far and w + ew >= far:
            continue                                 # too close to the clip planes to decide
        if not (near <= w < far):
            assert pixel[i] == -1
            checked += 1
            continue
        ok = True
        pix = []
        for c, tc, size in ((cx, tcx, view.width), (cy, tcy, view.height)):
            nd = c / w
            f = (nd / 2 + Fraction(1, 2)) * size
            # float rounding of clip values (2^-24 each), division, fma, multiply, plus FP64 error
            fp64 = (6 * u53 * tc + abs(nd) * ew) / w
            err = (abs(nd) * Fraction(8, 1 << 24) + Fraction(4, 1 << 24) + fp64) * size * 2
            fl = math.floor(f)
            if f - err < fl or f + err >= fl + 1:
                ok = False
            pix.append((f, fl))
        if not ok:
            continue
        (fx, px), (fy, py) = pix
        inside = 0 <= fx < view.width and 0 <= fy < view.height
        if not inside:
            assert pixel[i] == -1
            checked += 1
            continue
        assert pixel[i] == py * view.width + px, i
        t = (w - near) * s_exact
        et = s_exact * ew + 8 * u53 * abs(t)
        ft = math.floor(t)
        if t - et >= ft and t + et < ft + 1:
            assert int(q[i]) == min(ft, TWO40 - 2), (i, float(t), int(q[i]))
        checked += 1
    assert checked >= expect_checked, checked


def check_general_scene_against_exact_math():
    pts = scenes.cube(1500, 21)
    view = scenes.View.lookat((0.7, 0.4, 2.2), (0.02, -0.03, 0.01), (0.1, 1.0, 0.0), 55.0, 320, 200, 0.1, 10.0)
    _fp_bounds_check(pts, view, 1400)
    pts = scenes.lidar(1500, 22)
    _fp_bounds_check(pts, scenes.lidar_1km_view(480, 270), 1400)


# --------------------------------------------------------------------------------------------- HQ

def check_hq_band_inclusive():
    """Section 2.2: fragments at most 1 % deeper than the closest contribute. Metric mode (mm codes):
    closest w = 1 m -> q = 1000; bound 100 (q - 1000) <= 1000 -> q <= 1010 is inside, 1011 outside."""
    view = axis_view(8, 8, near=0.5, far=8.5, depth_mode=1, metric_scale=1000.0)
    ws = [1.0, 1.0107421875, 1.01171875, 1.005859375]  # q = 1000, 1010 (inclusive), 1011 (out), 1005 (in)
    cols = [rgba(10, 20, 30), rgba(20, 40, 61), rgba(200, 200, 200), rgba(0, 0, 0)]
    pts = pack([[0.0, 0.0, -w] for w in ws], cols)
    _, q, _ = oracle.project(pts, view)
    assert [int(v) for v in q] == [1000, 1010, 1011, 1005]
    fb = oracle.render_atomicmin(pts, view)
    (sr, sg, sb, cnt), ovf = oracle.hq_accumulate(pts, view, fb, 1, 100)
    pix = 4 * 8 + 4
    assert not ovf
    assert (int(sr[pix]), int(sg[pix]), int(sb[pix]), int(cnt[pix])) == (30, 60, 91, 3)
    img = oracle.resolve_hq((sr, sg, sb, cnt), background=0x12345678)
    assert int(img[pix]) == rgba(10, 20, 30)           # (30+1)/3, (60+1)/3, (91+1)/3
    assert int(np.count_nonzero(cnt)) == 1 and int(img[0]) == 0x12345678


def check_hq_average_rounding():
    """Average of (10,20,30) and (20,40,61) with round-half-up is (15,30,46); of (11,1,0) and (20,2,0)
    it is (16,2,0) (15.5 rounds up, 1.5 rounds up)."""
    view = axis_view(8, 8, near=0.5, far=8.5, depth_mode=1, metric_scale=1000.0)
    pts = pack([[0.0, 0.0, -1.0], [0.0, 0.0, -1.0], [0.25, 0.25, -1.0], [0.25, 0.25, -1.0]],
               [rgba(10, 20, 30), rgba(20, 40, 61), rgba(11, 1, 0), rgba(20, 2, 0)])
    fb = oracle.render_atomicmin(pts, view)
    acc, _ = oracle.hq_accumulate(pts, view, fb)
    img = oracle.resolve_hq(acc)
    assert int(img[4 * 8 + 4]) == rgba(15, 30, 46)
    assert int(img[5 * 8 + 5]) == rgba(16, 2, 0)


def check_hq_linear_band():
    """Linear mode: near 0.5, far 0.5 + 2^20 -> s = 2^20, Nq = near * s = 2^19; closest w = 1 (q = 2^19),
    so the band is q - qmin <= (qmin + Nq) / 100 = 2^20 / 100, i.e. depth up to 1.01 m. The depths
    below are float32 values, so every code is exact."""
    view = axis_view(8, 8, near=0.5, far=0.5 + 2.0 ** 20)
    bound_q = (1 << 19) + (1 << 20) // 100
    w_in = 1.0 + ((1 << 20) // 100) / 2.0 ** 20          # exactly at the inclusive bound
    w_out = 1.0 + ((1 << 20) // 100 + 1) / 2.0 ** 20
    pts = pack([[0.0, 0.0, -1.0], [0.0, 0.0, -w_in], [0.0, 0.0, -w_out]], [rgba(1, 1, 1), rgba(3, 3, 3), rgba(9, 9, 9)])
    _, q, _ = oracle.project(pts, view)
    assert [int(v) for v in q] == [1 << 19, bound_q, bound_q + 1]
    fb = oracle.render_atomicmin(pts, view)
    (sr, sg, sb, cnt), _ = oracle.hq_accumulate(pts, view, fb)
    pix = 4 * 8 + 4
    assert int(cnt[pix]) == 2 and int(sr[pix]) == 4


def check_hq_invariants():
    pts = scenes.lidar(30000, 7)
    view = scenes.lidar_1km_view(96, 54)
    fb = oracle.render_atomicmin(pts, view)
    (sr, sg, sb, cnt), ovf = oracle.hq_accumulate(pts, view, fb)
    assert not ovf
    assert np.array_equal(cnt > 0, fb != oracle.EMPTY)
    assert np.all(sr <= 255 * cnt) and np.all(sg <= 255 * cnt) and np.all(sb <= 255 * cnt)
    # with eps = 0 only fragments at exactly the closest depth code contribute; the winner always does
    (sr0, _, _, cnt0), _ = oracle.hq_accumulate(pts, view, fb, 0, 1)
    assert np.all(cnt0 <= cnt) and np.array_equal(cnt0 > 0, fb != oracle.EMPTY)


def check_resolve_basic():
    fb = np.array([oracle.EMPTY, (5 << 24) | 0x123456, (1 << 24) | 0xABCDEF, 0], np.uint64)
    img = oracle.resolve_basic(fb, background=0x01020304)
    assert img.tolist() == [0x01020304, 0xFF123456, 0xFFABCDEF, 0xFF000000]


def check_piecewise_ranges():
    """Section 2.1: [0, 10 m] in nanometres, [10 m, 10 km] in micrometres, [10 km, 10 000 km] in
    millimetres; each range takes at most 10 billion codes, about 30 billion in total."""
    with open(os.path.join(GOLDEN, "paper_piecewise_ranges.json")) as f:
        g = json.load(f)
    ranges = np.array([[r["lo_m"], r["hi_m"], r["codes_per_m"]] for r in g["ranges"]])
    view = axis_view(4, 4, near=1e-3, far=2e7, depth_mode=2)
    view.ranges = ranges
    ws = [0.5, 9.5, 10.0, 5000.0, 1e4, 1e6, 9.999e6, 1e7 + 1.0]
    pts = pack([[0.0, 0.0, -w] for w in ws], [0] * len(ws))
    pixel, q, _ = oracle.project(pts, view)
    counts = [math.ceil((r["hi_m"] - r["lo_m"]) * r["codes_per_m"]) for r in g["ranges"]]
    assert all(c <= g["max_codes_per_range"] for c in counts)
    assert sum(counts) <= g["approx_total_codes"]
    b1, b2 = counts[0], counts[0] + counts[1]
    assert int(q[0]) == 500_000_000 and int(q[1]) == 9_500_000_000
    assert int(q[2]) == b1 and int(q[3]) == b1 + math.floor((5000.0 - 10.0) * 1e6)
    assert int(q[4]) == b2 and int(q[5]) == b2 + math.floor((1e6 - 1e4) * 1e3)
    assert int(q[6]) == b2 + math.floor((9.999e6 - 1e4) * 1e3)
    assert pixel[7] == -1                         # beyond the last range
    assert int(q[6]) < TWO40 - 2


PINS = [check_exact_dyadic_linear, check_exact_dyadic_metric, check_frustum_edges, check_pixel_orientation,
        check_known_winners_and_tiebreak, check_empty_and_sentinel, check_depth_cap_and_capacity,
        check_paper_clear_value, check_bruteforce_tiny, check_order_invariance,
        check_general_scene_against_exact_math, check_hq_band_inclusive, check_hq_average_rounding,
        check_hq_linear_band, check_hq_invariants, check_resolve_basic, check_piecewise_ranges]


@pytest.mark.parametrize("check", PINS, ids=[c.__name__ for c in PINS])
def test_pin(check):
    check()


def test_invalid_views_rejected():
    pts = pack([[0, 0, -1.0]], [0])
    for bad in (axis_view(near=0.0), axis_view(near=2.0, far=1.0), axis_view(far=float("inf")),
                axis_view(depth_mode=1, metric_scale=0.0), axis_view(depth_mode=5)):
        with pytest.raises(ValueError):
            oracle.project(pts, bad)
