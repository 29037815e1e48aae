"""CPU restatement of the certified transform's first tier (csrc/pcr_certified.cuh: tier1_constants,
build_table, classify_fast) against the FP64 definition of the oracle (Sections 1 and 2.1).

The constants are restated from their derivation in FP64 and exact integers; the per-point arithmetic in IEEE
float32 with correctly rounded fused multiply-adds (the product of two floats is exact in float64, and a
float64 sum that lands on a float32 rounding midpoint is settled by the two-sum remainder); the 96-bit
fixed-point depth sum in exact integers. The approximate reciprocal of the kernel (rcp.approx, within one ulp)
is taken at both floats that bracket 1/w: whichever the hardware returns, every decision tier 1 takes must be
the definition's. On points chosen next to pixel edges, depth-code integers and clip planes (and on whole
scenes) each point that the restated tier 1 decides must get the oracle's pixel and code (or one of the two
neighbouring codes, when the code is left undecided), and each point it culls must be culled by the oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import scenes
from tests.helpers import axis_view, pack

F32 = np.float32
U = 2.0 ** -24
V53 = 2.0 ** -53
MAGIC = F32(12582912.0)  # 1.5 * 2^23


def f_up(x: float) -> np.float32:
    f = F32(x)
    return f if float(f) >= x else np.nextafter(f, F32(np.inf))


def f_down(x: float) -> np.float32:
    f = F32(x)
    return f if float(f) <= x else np.nextafter(f, F32(-np.inf))


def fma32(a, b, c):
    """RN32(a b + c), exact, for float32 arrays (finite, normal results)."""
    a64, b64, c64 = (np.asarray(v, np.float32).astype(np.float64) for v in (a, b, c))
    p = a64 * b64
    s = p + c64
    bb = s - p
    e = (p - (s - bb)) + (c64 - bb)
    with np.errstate(all="ignore"):
        r = s.astype(np.float32)
        t = r.astype(np.float64)
        up = np.nextafter(r, F32(np.inf)).astype(np.float64)
        dn = np.nextafter(r, F32(-np.inf)).astype(np.float64)
        # s on a float32 midpoint: between r and up (s > r) or dn and r (s < r)
        mid_hi = (s > t) & (s - t == up - s)
        mid_lo = (s < t) & (t - s == s - dn)
        r = np.where(mid_hi & (e > 0), np.nextafter(r, F32(np.inf)), r)
        r = np.where(mid_lo & (e < 0), np.nextafter(r, F32(-np.inf)), r)
    return r.astype(np.float32)


def add_ru(a, b):
    s = np.asarray(a, np.float32).astype(np.float64) + np.asarray(b, np.float32).astype(np.float64)
    with np.errstate(all="ignore"):
        r = s.astype(np.float32)
        return np.where(r.astype(np.float64) < s, np.nextafter(r, F32(np.inf)), r)


def add_rd(a, b):
    s = np.asarray(a, np.float32).astype(np.float64) + np.asarray(b, np.float32).astype(np.float64)
    with np.errstate(all="ignore"):
        r = s.astype(np.float32)
        return np.where(r.astype(np.float64) > s, np.nextafter(r, F32(-np.inf)), r)


def fma64(a: float, b: float, c: float) -> float:
    """RN64(a b + c), exact (float() of a Fraction rounds correctly)."""
    from fractions import Fraction
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def fixed_mul(a: float, b: float, k: int):
    """round(a b 2^k), ties away from zero, as the host code computes it; None when it reaches 2^126."""
    from fractions import Fraction
    if a == 0.0 or b == 0.0:
        return 0
    x = Fraction(a) * Fraction(b) * (Fraction(2) ** k)
    mag = (abs(x.numerator) * 2 + x.denominator) // (2 * x.denominator)
    if mag >= 1 << 126:
        return None
    return -mag if x < 0 else mag


class Tier1:
    """The first-tier constants of a LINEAR or METRIC view (tier1_constants and build_table restated)."""

    def __init__(self, view):
        m = np.asarray(view.view_proj, np.float64)
        self.W, self.H = view.width, view.height
        m0, m1, m3 = m[0], m[1], m[3]
        self.linear = getattr(view, "depth_mode", 0) == 0
        near, far = float(view.near), float(view.far)
        S = 1099511627776.0 / (far - near) if self.linear else float(getattr(view, "metric_scale", 1000.0))
        W, H = float(self.W), float(self.H)
        M = max(W, H)
        hw, hwm, hh, hhm = 0.5 * W, 0.5 * W - 0.5, 0.5 * H, 0.5 * H - 0.5
        gx = [fma64(hw, float(m0[c]), hwm * float(m3[c])) for c in range(4)]
        gy = [fma64(hh, float(m1[c]), hhm * float(m3[c])) for c in range(4)]
        self.Wr = [F32(m3[c]) for c in range(4)]
        self.Gx = [F32(g) for g in gx]
        self.Gy = [F32(g) for g in gy]
        m3max = max(abs(m3[c]) for c in range(3))
        hmax = max(max(hw * abs(m0[c]) + hwm * abs(m3[c]), hh * abs(m1[c]) + hhm * abs(m3[c])) for c in range(3))
        h3 = max(hw * abs(m0[3]) + hwm * abs(m3[3]), hh * abs(m1[3]) + hhm * abs(m3[3]))
        sl = (1.0 + 2.0001 * U) * (1.0 + 2.0 ** -20)
        self.Mw, self.Mw3 = f_up(m3max * sl), f_up(abs(m3[3]) * (1.0 + 2.0 ** -20))
        self.MH, self.MH3 = f_up(hmax * sl), f_up(h3 * (1.0 + 2.0 ** -20))
        t_lo, t_hi = 2.5, 1099511627776.0 - 33554432.0
        w_lo = near + t_lo / S if self.linear else t_lo / S
        w_hi = near + t_hi / S if self.linear else t_hi / S
        nin = max(near * (1.0 + 4.0 * U), w_lo * (1.0 + 4.0 * U))
        fin = min(far * (1.0 - 4.0 * U), w_hi * (1.0 - 4.0 * U))
        self.kw = f_up(4.0004 * U * float(self.Mw) * (1.0 + 2.0 ** -20))
        self.kw3 = f_up(4.0004 * U * float(self.Mw3) * (1.0 + 2.0 ** -20))
        self.wc = F32(0.5 * (nin + fin))
        wh = min(float(self.wc) - nin, fin - float(self.wc))
        whk = (wh - float(self.kw3)) / (1.0 + 2.0001 * U)
        self.whk = f_down(whk) if whk > 0 else F32(0.0)
        self.near_o, self.far_o = f_down(near), f_up(far)
        cE = 4.001 * U * (1.0 + 2.0 ** -19)
        self.ke = f_up(cE * (float(self.MH) + (M + 1.0) * float(self.Mw)))
        self.ke3 = f_up(cE * (float(self.MH3) + (M + 1.0) * float(self.Mw3)))
        self.he0 = f_down(0.5 - U * (6.51 * M + 3.51) - 2.0 ** -22 - 2.0 ** -24)
        self.cb = f_up(4.001 * U * (1.0 + 2.0 ** -19))
        self.ce = f_up(3.05 * U * max(hwm, hhm) + 2.0 ** -20)
        self.wm, self.hm = F32(W - 0.5), F32(H - 0.5)
        self.kd = f_up(5.2 * V53 * S * m3max * (1.0 + 2.0001 * U) * (1.0 + 2.0 ** -18))
        nl = near if self.linear else 0.0
        d0 = 5.2 * V53 * S * (abs(m3[3]) + nl) * (1.0 + 2.0 ** -18) + 3.1 * V53 * S * nl + 2.0 ** -13
        self.hd0 = f_down(0.5 - d0 - 2.0 ** -22)
        # the depth table: F[j][e] = round(S M3_j 2^(e - 150 + 40)), e_max[j] the largest usable exponent
        self.F = np.zeros((3, 256), dtype=object)
        e_max = []
        for j in range(3):
            em = 254
            for e in range(256):
                ee = 1 if e == 0 else e
                f = fixed_mul(S, m3[j], ee - 150 + 40) if e < 255 else None
                if f is None or not (-(1 << 62) < f < (1 << 62)):
                    em = min(em, e - 1)
                    f = 0
                self.F[j][e] = f
            e_max.append(em)
        b = fixed_mul(S, m3[3], 40) - (fixed_mul(S, near, 40) if self.linear else 0)
        self.B = b
        emin = min(e_max)
        self.xyz_max = F32(3.0e38) if emin >= 254 else F32(2.0 ** min(127, emin - 127 + 1))

    def classify(self, pts: np.ndarray, r_variant: int):
        """The kernel's tier 1 on (n, 4) uint32 points with the reciprocal rounded down (r_variant 0) or up (1).
        Returns state (0 culled, 1 exact, 2 code undecided, 4 deferred), pixel and the code floor qc."""
        bits = pts[:, :3].astype(np.uint32)
        xyz = bits.view(np.float32)
        x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
        with np.errstate(all="ignore"):
            s = (np.abs(x) + np.abs(y)) + np.abs(z)
            in_range = s < self.xyz_max
            w = fma32(self.Wr[2], z, fma32(self.Wr[1], y, fma32(self.Wr[0], x, self.Wr[3])))
            depth_in = np.abs(w - self.wc) < fma32(-self.kw, s, self.whk)
            # depth code: the 96-bit fixed-point sum, as the kernel accumulates it (low and high 32-bit halves)
            L = np.full(len(pts), self.B & 0xFFFFFFFF, dtype=object)
            Hh = np.full(len(pts), self.B >> 32, dtype=object)
            for j in range(3):
                idx = (bits[:, j] >> 23).astype(np.int64)
                sign = idx >> 8
                f = np.array([self.F[j][e & 0xFF] for e in idx], dtype=object)
                f = np.where(sign == 1, -f, f)
                mj = ((bits[:, j] & 0x7FFFFF) | 0x800000).astype(np.int64).astype(object)
                L = L + mj * (f & 0xFFFFFFFF)
                Hh = Hh + mj * (f >> 32)
            t_hi = (L >> 32) + Hh  # t * 2^40 = t_hi * 2^32 + (L mod 2^32)
            a0 = L & 0xFFFFFFFF
            a1 = t_hi & 0xFFFFFFFF
            frac_bits = np.array([((int(h) << 32 | int(lo)) >> 17) & 0x7FFFFF for h, lo in zip(a1, a0)], np.int64)
            frac = (frac_bits.astype(np.float64) / 2.0 ** 23).astype(np.float32)
            qc = np.array([int(h) >> 8 for h in t_hi], dtype=np.int64)
            hD = fma32(-self.kd, s, self.hd0)
            exact = np.abs(frac - F32(0.5)) < hD
            amb_ok = hD > F32(0.25)
            gx = fma32(self.Gx[2], z, fma32(self.Gx[1], y, fma32(self.Gx[0], x, self.Gx[3])))
            gy = fma32(self.Gy[2], z, fma32(self.Gy[1], y, fma32(self.Gy[0], x, self.Gy[3])))
            r64 = 1.0 / w.astype(np.float64)
            r = r64.astype(np.float32)
            lo = np.where(r.astype(np.float64) > r64, np.nextafter(r, F32(-np.inf)), r)
            hi = np.where(r.astype(np.float64) < r64, np.nextafter(r, F32(np.inf)), r)
            r = lo if r_variant == 0 else hi
            fxm, fym = (gx * r).astype(np.float32), (gy * r).astype(np.float32)
            hE = fma32(-fma32(self.ke, s, self.ke3), r, self.he0)
            gxx, gyy = (fxm + MAGIC).astype(np.float32), (fym + MAGIC).astype(np.float32)
            kx = (gxx.view(np.int32).astype(np.int64) - 0x4B400000) & 0xFFFFFFFF
            ky = (gyy.view(np.int32).astype(np.int64) - 0x4B400000) & 0xFFFFFFFF
            dx = (fxm - (gxx - MAGIC)).astype(np.float32)
            dy = (fym - (gyy - MAGIC)).astype(np.float32)
            ax_ok = (kx < self.W) & (ky < self.H) & (np.abs(dx) < hE) & (np.abs(dy) < hE)
            visible = in_range & depth_in & ax_ok & (exact | amb_ok)
            dw = fma32(self.kw, s, self.kw3)
            depth_out = (add_ru(w, dw) < self.near_o) | (add_rd(w, -dw) >= self.far_o)
            bf = ((fma32(self.Mw, s, self.Mw3) * r).astype(np.float32) * self.cb).astype(np.float32)
            gf = ((fma32(self.MH, s, self.MH3) * r).astype(np.float32) * self.cb).astype(np.float32)
            ea, eb = fma32(F32(1.35), bf, F32(9.8 * U)), fma32(F32(1.35), gf, self.ce)
            ex, ey = fma32(np.abs(fxm), ea, eb), fma32(np.abs(fym), ea, eb)
            ax_out = (fxm < -add_ru(F32(0.5), ex)) | (fxm >= add_ru(self.wm, ex)) | \
                (fym < -add_ru(F32(0.5), ey)) | (fym >= add_ru(self.hm, ey))
            e_finite = (ex + ey).astype(np.float32) < F32(3.0e38)
            culled = in_range & (depth_out | (depth_in & (bf <= F32(0.25)) & e_finite & ax_out))
        state = np.where(visible, np.where(exact, 1, 2), np.where(culled, 0, 4))
        pixel = ky * self.W + kx
        return state, pixel, qc, frac


def _check_view(pts, view, min_decided=0.9):
    o_pix, _, o_key = oracle.project(pts, view)
    o_code = np.where(o_pix >= 0, (o_key >> np.uint64(24)).astype(np.int64), -1)
    t = Tier1(view)
    for variant in (0, 1):
        state, pixel, qc, frac = t.classify(pts, variant)
        ex = state == 1
        bad = ex & ((o_pix != pixel) | (o_code != qc))
        assert not bad.any(), ("exact", variant, np.flatnonzero(bad)[:5])
        am = state == 2
        lo = frac < F32(0.5)
        cand_ok = np.where(lo, (o_code == qc - 1) | (o_code == qc), (o_code == qc) | (o_code == qc + 1))
        bad = am & ((o_pix != pixel) | ~cand_ok)
        assert not bad.any(), ("undecided code", variant, np.flatnonzero(bad)[:5])
        bad = (state == 0) & (o_pix >= 0)
        assert not bad.any(), ("culled", variant, np.flatnonzero(bad)[:5])
        decided = np.mean(state != 4)
        assert decided >= min_decided, (variant, decided)
    return state


def _near_boundary(view, n, seed):
    """Points in front of the camera whose depth code, pixel coordinate or clip x lies next to a decision
    boundary of the definition, found with numpy FP64 (the same selection as the GPU parity tests)."""
    from tests.test_gpu_parity import _near_boundary_points
    pts, _ = _near_boundary_points(view, n, seed)
    return pts


def _near_clip_planes(view, n, seed):
    """Points whose depth w lies within a few parts in 10^6 of the near or the far plane, at random ndc."""
    rng = np.random.default_rng(seed)
    M = np.asarray(view.view_proj, dtype=np.float64)
    inv = np.linalg.inv(M)
    ndc = rng.uniform(-1.0, 1.0, (n, 2))
    plane = np.where(rng.random(n) < 0.5, view.near, view.far)
    w = plane * (1.0 + rng.uniform(-4e-6, 4e-6, n))
    f_, n_ = view.far, view.near
    zc = (f_ + n_) / (f_ - n_) * w + 2.0 * f_ * n_ / (n_ - f_)
    world = np.stack([ndc[:, 0] * w, ndc[:, 1] * w, zc, w], 1) @ inv.T
    xyz = (world[:, :3] / world[:, 3:4]).astype(np.float32)
    return pack(xyz, rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32))


def test_lidar_view_boundary_points():
    view = scenes.lidar_1km_view(640, 360)
    pts = _near_boundary(view, 2_000_000, 11)
    assert len(pts) > 5000
    _check_view(pts, view, 0.5)


def test_clip_planes():
    for view in (scenes.lidar_1km_view(640, 360), scenes.cube_1m_view()):
        pts = _near_clip_planes(view, 40_000, 17)
        state = _check_view(pts, view, 0.0)
        # tier 1 leaves the points nearest the planes to tier 2 and decides (keeps or culls) the others
        assert 0.01 < np.mean(state == 4) < 0.9, np.mean(state == 4)


def test_lidar_scene_and_culling():
    view = scenes.lidar_1km_view(800, 450)
    pts = scenes.lidar(200_000, 12)
    state = _check_view(pts, view, 0.95)
    assert np.mean(state == 1) > 0.9


def test_cube_and_camera_inside_the_cloud():
    _check_view(scenes.cube(100_000, 13), scenes.cube_1m_view(), 0.95)
    rng = np.random.default_rng(14)
    xyz = rng.normal(0.0, 3.0, (100_000, 3))  # the camera sits inside: points behind, beside, in front
    view = scenes.View.lookat((0.0, 0.0, 0.0), (1.0, 0.3, -0.2), (0.0, 0.0, 1.0), 75.0, 333, 211, 0.05, 20.0)
    _check_view(pack(xyz, np.arange(100_000, dtype=np.uint32)), view, 0.8)


def test_metric_depth_and_axis_views():
    base = scenes.lidar_1km_view(512, 288)
    v = scenes.View(base.view_proj, base.near, base.far, 512, 288)
    v.depth_mode = 1
    v.metric_scale = 1000.0
    _check_view(_near_boundary(base, 200_000, 15), v, 0.5)
    av = axis_view(64, 48)
    rng = np.random.default_rng(16)
    xyz = np.column_stack([rng.uniform(-6, 6, 50_000), rng.uniform(-6, 6, 50_000), rng.uniform(-9, 0, 50_000)])
    _check_view(pack(xyz, np.zeros(50_000, np.uint32)), av, 0.8)
