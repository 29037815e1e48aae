// Per-point transform without a framebuffer (pcr_project_points in include/pcr.h): for every point, the pixel
// and the key the definition of Sections 1 and 2.1 gives it, or 0xFFFFFFFF and the empty key when it is culled.
// Not a hot path: one point per thread, plain loads, no staging. It exposes, point by point, the same
// decisions the raster passes take (tier 1, tier 2, FP64 arbiter), so they can be checked against the
// definition for every point and not only for the fragments that win a pixel.
#pragma once

#include "pcr_certified.cuh"

namespace pcr {

// EXACT (kApprox = false): tier 1 decides nearly every point; a point it cannot decide goes through tier 2
// and, if that cannot decide either, through the FP64 definition. DOUBLE_FLOAT (kApprox = true): the
// double-float evaluation alone. The depth table is read from the kernel parameter block; kPw (PIECEWISE
// depth): the ranges' tables from the device copy `table` into dynamic shared memory.
template <bool kApprox, int kPw = 0>
__global__ void __launch_bounds__(256) k_project_cert(const uint4* __restrict__ pts, uint64_t n,
                                                      const __grid_constant__ CertParams P,
                                                      uint32_t* __restrict__ pix_out,
                                                      unsigned long long* __restrict__ key_out,
                                                      const long long* __restrict__ table = nullptr) {
  __shared__ long long sF_static[kPw ? 1 : 3 * kTableEntries];
  extern __shared__ __align__(16) long long sF_dynamic[];
  long long* const sF = kPw ? sF_dynamic : sF_static;
  if constexpr (kPw) {
    for (int i = threadIdx.x; i < P.n_pw * 3 * kTableEntries; i += blockDim.x) sF[i] = table[i];
    __syncthreads();
  } else if (!kApprox) {
    load_table(P, sF);
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 p = pts[i];
    uint32_t pix = 0xFFFFFFFFu;
    unsigned long long key = kEmptyKey;
    if (kApprox) {
      const CertFrag f = classify_df(P, p);
      if (f.state == kExact) {
        pix = f.pixel;
        key = make_key((unsigned long long)f.q, p.w);
      }
    } else {
      const FastFrag f = classify_fast<CertParams, kPw>(P, sF, p);
      if (f.state == kExact) {
        pix = f.pixel;
        key = key_from_fixed(f.a0, f.a1, f.a2, p.w);
      } else if (f.state != kCulled) {
        const CertFrag c = classify_cert(P, sF, p);
        if (c.state == kExact) {
          pix = c.pixel;
          key = make_key((unsigned long long)c.q, p.w);
        } else if (c.state != kCulled) {
          uint32_t px;
          unsigned long long q;
          if (project_fp64(P.v, __uint_as_float(p.x), __uint_as_float(p.y), __uint_as_float(p.z), &px, &q)) {
            pix = px;
            key = make_key(q, p.w);
          }
        }
      }
    }
    pix_out[i] = pix;
    key_out[i] = key;
  }
}

// FP64 (and every view outside the single-precision preconditions, piecewise depth included): each point
// through the FP64 definition directly.
__global__ void __launch_bounds__(256) k_project_fp64(const uint4* __restrict__ pts, uint64_t n, const DevView v,
                                                      uint32_t* __restrict__ pix_out,
                                                      unsigned long long* __restrict__ key_out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 p = pts[i];
    uint32_t px;
    unsigned long long q;
    const bool vis = project_fp64(v, __uint_as_float(p.x), __uint_as_float(p.y), __uint_as_float(p.z), &px, &q);
    pix_out[i] = vis ? px : 0xFFFFFFFFu;
    key_out[i] = vis ? make_key(q, p.w) : kEmptyKey;
  }
}

}  // namespace pcr
