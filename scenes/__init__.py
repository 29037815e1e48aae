"""Seeded synthetic scenes and cameras: the inputs shared by the oracle tests, the CUDA parity tests and
the benchmark.

The paper's scanned data sets (Heidentor 26M, Retz 145M/120M, Morro Bay 117M points; Table 1) are not
available, so these generators stand in for them at their scale and structure: a uniform cube, and a
LIDAR-like scene (sin-sum heightfield terrain + box buildings, centimetre noise, height-ramp colours,
coherent scan order, optional shuffled order to expose the order sensitivity noted in Section 3).

Nothing here projects, quantises or packs keys: this module only produces points (16 B each: float32
x, y, z + RGBA8 with byte 0 = R) and 4x4 view-projection matrices.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scenes.cpp")
_LIB_PATH = os.path.join(_HERE, "libpcrscenes.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library in place (g++, no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                               "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class LidarParams(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("amp_scale", ctypes.c_double), ("wavelength_scale", ctypes.c_double),
                ("n_boxes", ctypes.c_int32),
                ("box_fp_min", ctypes.c_double), ("box_fp_max", ctypes.c_double),
                ("box_h_min", ctypes.c_double), ("box_h_max", ctypes.c_double),
                ("noise_sigma", ctypes.c_double),
                ("street_x", ctypes.c_double), ("street_y", ctypes.c_double),
                ("street_radius", ctypes.c_double), ("street_fraction", ctypes.c_double),
                ("box_exclusion", ctypes.c_double)]


def lidar_params_1km() -> LidarParams:
    """1 km x 1 km terrain with 200 buildings (footprint 10-40 m, height 5-60 m), 1 cm noise."""
    return LidarParams(0.0, 1000.0, 0.0, 1000.0, 1.0, 1.0, 200, 10.0, 40.0, 5.0, 60.0, 0.01,
                       0.0, 0.0, 0.0, 0.0, 0.0)


def lidar_params_city() -> LidarParams:
    """10 km x 10 km city ([-5000, 5000]^2) with 8000 buildings and street-level detail within 20 m of
    the origin, so that points a few centimetres from a street-level eye exist."""
    return LidarParams(-5000.0, 5000.0, -5000.0, 5000.0, 0.25, 10.0, 8000, 10.0, 40.0, 5.0, 60.0, 0.01,
                       0.0, 0.0, 20.0, 0.02, 30.0)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.scn_gen_cube.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int]
        lib.scn_gen_lidar.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(LidarParams), ctypes.c_void_p,
                                      ctypes.c_int]
        lib.scn_lidar_height.argtypes = [ctypes.c_uint64, ctypes.POINTER(LidarParams), ctypes.c_double, ctypes.c_double]
        lib.scn_lidar_height.restype = ctypes.c_double
        lib.scn_shuffle.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]
        lib.scn_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.scn_splitmix64_at.restype = ctypes.c_uint64
        _lib = lib
    return _lib


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def _out(n: int, out):
    if out is None:
        return np.empty((n, 4), dtype=np.uint32), None
    # Any buffer exposing a data pointer of n * 16 bytes (numpy array or pinned CPU torch tensor).
    ptr = out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()
    return out, ptr


def splitmix64_at(state: int, n: int) -> int:
    """n-th output of the SplitMix64 sequence started at `state` (exported for its known-answer test)."""
    return int(_load().scn_splitmix64_at(state, n))


def cube(n: int, seed: int = 1, half: float = 0.5, out=None, threads: int | None = None):
    """n points uniform in [-half, half]^3 with three random colour bytes and alpha 255."""
    arr, ptr = _out(n, out)
    rc = _load().scn_gen_cube(n, seed, half, ptr if ptr is not None else arr.ctypes.data, threads or _threads())
    if rc != 0:
        raise RuntimeError("scn_gen_cube failed")
    return arr


def lidar(n: int, seed: int, params: LidarParams | None = None, out=None, threads: int | None = None):
    """n points of the LIDAR-like scene, coherent order (terrain strips, then buildings, then street)."""
    params = params or lidar_params_1km()
    arr, ptr = _out(n, out)
    rc = _load().scn_gen_lidar(n, seed, ctypes.byref(params), ptr if ptr is not None else arr.ctypes.data,
                               threads or _threads())
    if rc != 0:
        raise RuntimeError("scn_gen_lidar failed")
    return arr


def lidar_height(seed: int, params: LidarParams, x: float, y: float) -> float:
    return float(_load().scn_lidar_height(seed, ctypes.byref(params), x, y))


def shuffle(points, seed: int):
    """Seeded in-place Fisher-Yates shuffle of a point array (numpy (n, 4) uint32 or CPU torch tensor)."""
    n = points.shape[0]
    ptr = points.ctypes.data if isinstance(points, np.ndarray) else points.data_ptr()
    if _load().scn_shuffle(ptr, n, seed) != 0:
        raise RuntimeError("scn_shuffle failed")
    return points


# ----------------------------------------------------------------------------------------------- cameras

def look_at(eye, target, up) -> np.ndarray:
    """World-to-view matrix (row-major, column vectors), camera looking down its -z axis."""
    eye, target, up = (np.asarray(v, dtype=np.float64) for v in (eye, target, up))
    f = target - eye
    f = f / math.sqrt(float(f @ f))
    s = np.cross(f, up)
    s = s / math.sqrt(float(s @ s))
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    m[0, 3], m[1, 3], m[2, 3] = -(s @ eye), -(u @ eye), f @ eye
    return m


def perspective(fovy_deg: float, aspect: float, near: float, far: float) -> np.ndarray:
    """OpenGL-style perspective projection; clip w = -z_view, the distance along the view axis."""
    f = 1.0 / math.tan(math.radians(fovy_deg) * 0.5)
    m = np.zeros((4, 4))
    m[0, 0] = f / aspect
    m[1, 1] = f
    m[2, 2] = (far + near) / (near - far)
    m[2, 3] = 2.0 * far * near / (near - far)
    m[3, 2] = -1.0
    return m


@dataclass
class View:
    """A camera: row-major 4x4 view-projection (clip = M @ (x, y, z, 1)), clip range, depth mapping."""
    view_proj: np.ndarray
    near: float
    far: float
    width: int
    height: int
    depth_mode: int = 0          # 0: linear [near, far) -> [0, 2^40); 1: metric floor(w * metric_scale)
    metric_scale: float = 1000.0

    @staticmethod
    def lookat(eye, target, up, fovy_deg, width, height, near, far, **kw) -> "View":
        vp = perspective(fovy_deg, width / height, near, far) @ look_at(eye, target, up)
        return View(np.ascontiguousarray(vp, dtype=np.float64), float(near), float(far), int(width), int(height), **kw)


def orbit_views(count: int, seed: int, centre=(500.0, 500.0, 0.0), resolutions=((640, 480), (1920, 1080), (3840, 2160)),
                near: float = 0.1, far: float = 3000.0) -> list[View]:
    """Seeded orbit poses: azimuth U[0, 2pi), elevation U[15, 75] deg, radius U[300, 1500] m, target
    jittered by +-100 m around `centre`; resolutions cycle through `resolutions` by pose index."""
    views = []
    for i in range(count):
        r = [splitmix64_at(seed * 0x100000001B3 + 77, 6 * i + k) for k in range(5)]
        u = [(x >> 11) * (1.0 / 9007199254740992.0) for x in r]
        az = 2.0 * math.pi * u[0]
        el = math.radians(15.0 + 60.0 * u[1])
        rad = 300.0 + 1200.0 * u[2]
        tgt = np.array([centre[0] + (u[3] * 2 - 1) * 100.0, centre[1] + (u[4] * 2 - 1) * 100.0, centre[2]])
        eye = tgt + rad * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        w, h = resolutions[i % len(resolutions)]
        views.append(View.lookat(eye, tgt, (0.0, 0.0, 1.0), 60.0, w, h, near, far))
    return views


# ------------------------------------------------------------------------------------ named workloads

def cube_1m_view() -> View:
    """1M-point unit cube workload camera: 640x480, fov 60 deg, near 0.1, far 10, eye (0,0,3) -> origin."""
    return View.lookat((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, 640, 480, 0.1, 10.0)


def lidar_1km_view(width: int = 1920, height: int = 1080, **kw) -> View:
    """LIDAR 1 km workload camera: eye (-150,-150,350) looking at (500,500,0), z up, fov 60, near 0.1, far 3000."""
    return View.lookat((-150.0, -150.0, 350.0), (500.0, 500.0, 0.0), (0.0, 0.0, 1.0), 60.0, width, height, 0.1, 3000.0, **kw)


def city_view(seed: int = 4, width: int = 3840, height: int = 2160) -> View:
    """Street-level camera for the city scene: 1.7 m above the terrain at the origin, looking along +x
    (slightly to the side), fov 60, near 0.01, far 10000."""
    p = lidar_params_city()
    z = lidar_height(seed, p, 0.0, 0.0) + 1.7
    return View.lookat((0.0, 0.0, z), (100.0, 37.0, z), (0.0, 0.0, 1.0), 60.0, width, height, 0.01, 10000.0)
