"""GB300-native point-cloud rasterizer (atomicMin with 40-bit FP64 depth codes, high-quality splatting)
after Schuetz & Wimmer, "Rendering Point Clouds with Compute Shaders" (arXiv 1908.02681).

The compute path is the CUDA library `libpcr.so` (C ABI in include/pcr.h); `pcr` is its Python binding.
"""
from . import pcr  # noqa: F401
