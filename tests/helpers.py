"""Small helpers shared by the tests: point packing and exact-view construction (no rasterizer arithmetic)."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def pack(xyz, rgba) -> np.ndarray:
    """(n, 3) float32 coordinates + n RGBA8 words -> (n, 4) uint32 points."""
    xyz = np.asarray(xyz, dtype=np.float32).reshape(-1, 3)
    out = np.empty((xyz.shape[0], 4), np.uint32)
    out[:, :3] = xyz.view(np.uint32)
    out[:, 3] = np.asarray(rgba, dtype=np.uint32).reshape(-1)
    return out


def rgba(r, g, b, a=255) -> int:
    return (r & 0xFF) | ((g & 0xFF) << 8) | ((b & 0xFF) << 16) | ((a & 0xFF) << 24)


@dataclass
class RawView:
    """A view given directly by its matrix (tests build exact dyadic matrices by hand)."""
    view_proj: np.ndarray
    near: float
    far: float
    width: int
    height: int
    depth_mode: int = 0
    metric_scale: float = 1000.0
    ranges: np.ndarray | None = None
    transform: int = 0


def axis_view(width=64, height=48, near=0.5, far=8.5, **kw) -> RawView:
    """Camera at the origin looking down -z with clip x = x, clip y = y, w = -z (so ndc = (x/w, y/w))."""
    m = np.zeros((4, 4))
    m[0, 0] = 1.0
    m[1, 1] = 1.0
    m[2, 2] = -1.0
    m[3, 2] = -1.0
    return RawView(m, near, far, width, height, **kw)
