// Device-side definitions shared by the libpcr kernels: the per-view constants, the 16-byte streaming
// point load, and the FP64 per-point transform (the definition of Sections 1 and 2.1 of arXiv
// 1908.02681, evaluated with explicitly rounded operations so that no contraction changes a result).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pcr {

constexpr unsigned long long kEmptyKey = 0xFFFFFFFFFFFFFFFFull;
constexpr unsigned long long kQMax = (1ull << 40) - 2;  // largest depth code: no key can equal kEmptyKey
constexpr int kMaxRanges = 8;

enum : uint32_t { kStatusOverflow = 1u, kStatusTimeout = 2u };

// Per-view constants, passed by value as a kernel parameter.
struct DevView {
  double m[12];  // rows 0, 1 and 3 of the row-major view-projection: clip x, clip y, w
  double near_, far_;
  double scale;  // LINEAR: s = 2^40 / (far - near) (FP64, rounded once); METRIC: metric_scale
  double lo[kMaxRanges], hi[kMaxRanges], res[kMaxRanges], base[kMaxRanges];  // PIECEWISE
  unsigned long long nq;  // HQ: depth code of the near plane, floor(near * s) (LINEAR) or 0
  float fwidth, fheight;  // (float)W, (float)H
  int32_t width, height;
  int32_t depth_mode, n_ranges;
};

// 16-byte streaming load (each point is read once per pass): not allocated in L1; with PCR_LOAD_CS the
// streaming policy (evict first) in both levels, so the stream does not displace the framebuffer in L2.
__device__ __forceinline__ uint4 ld_stream16(const uint4* p) {
  uint4 v;
#ifdef PCR_LOAD_CS
  asm volatile("ld.global.cs.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
#else
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
#endif
  return v;
}

// Depth code of a visible fragment from its FP64 depth w (Section 2.1). Returns false when the
// piecewise mapping has no range for w.
__device__ __forceinline__ bool depth_code_fp64(const DevView& v, double w, unsigned long long* q) {
  double t;
  if (v.depth_mode == 0) {
    t = __dmul_rn(__dsub_rn(w, v.near_), v.scale);
  } else if (v.depth_mode == 1) {
    t = __dmul_rn(w, v.scale);
  } else {
    int k = 0;
    for (; k < v.n_ranges; ++k)
      if (w >= v.lo[k] && w < v.hi[k]) break;
    if (k == v.n_ranges) return false;
    t = __dadd_rn(v.base[k], floor(__dmul_rn(__dsub_rn(w, v.lo[k]), v.res[k])));
  }
  const double ft = floor(t);
  *q = ft >= (double)kQMax ? kQMax : __double2ull_rz(ft);
  return true;
}

// The FP64 transform of one point: true when visible, with its pixel index and depth code.
__device__ __forceinline__ bool project_fp64(const DevView& v, float x, float y, float z, uint32_t* pixel,
                                             unsigned long long* q) {
  const double X = x, Y = y, Z = z;
  const double cx = __fma_rn(v.m[2], Z, __fma_rn(v.m[1], Y, __fma_rn(v.m[0], X, v.m[3])));
  const double cy = __fma_rn(v.m[6], Z, __fma_rn(v.m[5], Y, __fma_rn(v.m[4], X, v.m[7])));
  const double w = __fma_rn(v.m[10], Z, __fma_rn(v.m[9], Y, __fma_rn(v.m[8], X, v.m[11])));
  if (!(w >= v.near_ && w < v.far_)) return false;
  const float fw = __double2float_rn(w), fcx = __double2float_rn(cx), fcy = __double2float_rn(cy);
  const float fx = __fmul_rn(__fmaf_rn(__fdiv_rn(fcx, fw), 0.5f, 0.5f), v.fwidth);
  const float fy = __fmul_rn(__fmaf_rn(__fdiv_rn(fcy, fw), 0.5f, 0.5f), v.fheight);
  if (!(fx >= 0.0f && fx < v.fwidth && fy >= 0.0f && fy < v.fheight)) return false;
  if (!depth_code_fp64(v, w, q)) return false;
  *pixel = (uint32_t)__float2int_rz(fy) * (uint32_t)v.width + (uint32_t)__float2int_rz(fx);
  return true;
}

__device__ __forceinline__ unsigned long long make_key(unsigned long long q, uint32_t rgba) {
  return (q << 24) | (unsigned long long)(rgba & 0xFFFFFFu);
}

// HQ band test (Section 2.2), exact on integers: eps_den * (q - qmin) <= eps_num * (qmin + Nq).
__device__ __forceinline__ bool in_band(unsigned long long q, unsigned long long qmin, unsigned long long nq,
                                        uint32_t eps_num, uint32_t eps_den) {
  return (unsigned long long)eps_den * (q - qmin) <= (unsigned long long)eps_num * (qmin + nq);
}

// Packed HQ increments: {R | G << 32} and {B | 1 << 32}.
__device__ __forceinline__ unsigned long long hq_rg(uint32_t rgba) {
  return (unsigned long long)(rgba & 0xFFu) | ((unsigned long long)((rgba >> 8) & 0xFFu) << 32);
}
__device__ __forceinline__ unsigned long long hq_bc(uint32_t rgba) {
  return (unsigned long long)((rgba >> 16) & 0xFFu) | (1ull << 32);
}

}  // namespace pcr
