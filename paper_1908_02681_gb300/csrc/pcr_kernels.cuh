// Per-pixel kernels (clear, resolves) and the FP64 per-point kernels of libpcr.
#pragma once

#include "pcr_device.cuh"

namespace pcr {

// Section 2.1 clear value: keys -> empty; HQ sums and counts -> 0. Two pixels per thread per step
// (16-byte stores); grid-stride.
__global__ void k_clear(unsigned long long* __restrict__ keys, ulonglong2* __restrict__ accum, uint64_t npx) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t pairs = npx >> 1;
  ulonglong2* k2 = reinterpret_cast<ulonglong2*>(keys);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < pairs; i += stride) {
    k2[i] = make_ulonglong2(kEmptyKey, kEmptyKey);
    if (accum) {
      accum[2 * i] = make_ulonglong2(0ull, 0ull);
      accum[2 * i + 1] = make_ulonglong2(0ull, 0ull);
    }
  }
  if ((npx & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    keys[npx - 1] = kEmptyKey;
    if (accum) accum[npx - 1] = make_ulonglong2(0ull, 0ull);
  }
}

// Section 2.1 with every point through the FP64 transform: one atomic minimum per visible fragment.
__global__ void __launch_bounds__(256) k_raster_fp64(const uint4* __restrict__ pts, uint64_t n, DevView v,
                                                     unsigned long long* __restrict__ keys) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 p = ld_stream16(pts + i);
    uint32_t pix;
    unsigned long long q;
    if (project_fp64(v, __uint_as_float(p.x), __uint_as_float(p.y), __uint_as_float(p.z), &pix, &q))
      atomicMin(keys + pix, make_key(q, p.w));
  }
}

// Section 2.2, second pass, FP64 transform: fragments within the depth band of their pixel's closest
// fragment add (R, G, B) and 1 to the pixel's sums.
__global__ void __launch_bounds__(256) k_hq_fp64(const uint4* __restrict__ pts, uint64_t n, DevView v,
                                                 const unsigned long long* __restrict__ keys,
                                                 unsigned long long* __restrict__ accum, uint32_t eps_num,
                                                 uint32_t eps_den) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 p = ld_stream16(pts + i);
    uint32_t pix;
    unsigned long long q;
    if (!project_fp64(v, __uint_as_float(p.x), __uint_as_float(p.y), __uint_as_float(p.z), &pix, &q)) continue;
    const unsigned long long qmin = keys[pix] >> 24;
    if (in_band(q, qmin, v.nq, eps_num, eps_den)) {
      atomicAdd(accum + 2 * (uint64_t)pix, hq_rg(p.w));
      atomicAdd(accum + 2 * (uint64_t)pix + 1, hq_bc(p.w));
    }
  }
}

// Section 2.1 resolve: key -> RGBA8 (alpha 255), background where empty; optional clear (keys, and the
// HQ sums when present).
__global__ void k_resolve_basic(unsigned long long* __restrict__ keys, ulonglong2* __restrict__ accum,
                                uint32_t* __restrict__ rgba, uint64_t npx, uint32_t background, int clear) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npx; i += stride) {
    const unsigned long long k = keys[i];
    rgba[i] = k == kEmptyKey ? background : ((uint32_t)(k & 0xFFFFFFu) | 0xFF000000u);
    if (clear) {
      keys[i] = kEmptyKey;
      if (accum) accum[i] = make_ulonglong2(0ull, 0ull);
    }
  }
}

// Section 2.2 third pass: per channel (sum + count / 2) / count, alpha 255, background where count is 0.
// A count above 2^24 means a u32 colour sum may have wrapped: flagged in the status word.
__global__ void k_resolve_hq(ulonglong2* __restrict__ accum, unsigned long long* __restrict__ keys,
                             uint32_t* __restrict__ rgba, uint64_t npx, uint32_t background, int clear,
                             uint32_t* __restrict__ status) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  bool overflow = false;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npx; i += stride) {
    const ulonglong2 a = accum[i];
    const uint32_t c = (uint32_t)(a.y >> 32);
    if (c == 0) {
      rgba[i] = background;
    } else if (c <= (1u << 24)) {
      // each channel sum is at most 255 c, so sum + c / 2 < 2^32: the 32-bit quotient is the same
      const uint32_t h = c / 2;
      const uint32_t r = ((uint32_t)a.x + h) / c;
      const uint32_t g = ((uint32_t)(a.x >> 32) + h) / c;
      const uint32_t b = ((uint32_t)a.y + h) / c;
      rgba[i] = (r & 0xFFu) | ((g & 0xFFu) << 8) | ((b & 0xFFu) << 16) | 0xFF000000u;
    } else {  // more fragments than the sums can hold: flagged; the same arithmetic as the oracle's, in 64 bits
      overflow = true;
      const uint32_t r = (uint32_t)(((a.x & 0xFFFFFFFFull) + c / 2) / c);
      const uint32_t g = (uint32_t)(((a.x >> 32) + c / 2) / c);
      const uint32_t b = (uint32_t)(((a.y & 0xFFFFFFFFull) + c / 2) / c);
      rgba[i] = (r & 0xFFu) | ((g & 0xFFu) << 8) | ((b & 0xFFu) << 16) | 0xFF000000u;
    }
    if (clear) {
      accum[i] = make_ulonglong2(0ull, 0ull);
      keys[i] = kEmptyKey;
    }
  }
  if (overflow) atomicOr(status, kStatusOverflow);
}

// Both resolves of an HQ frame in one pass over the pixels (Section 2.1 from the keys, Section 2.2 from the
// sums): each pixel's key and sums are read once and both images written, the same values as k_resolve_basic
// and k_resolve_hq; optional clear of both buffers.
__global__ void k_resolve_both(unsigned long long* __restrict__ keys, ulonglong2* __restrict__ accum,
                               uint32_t* __restrict__ rgba_basic, uint32_t* __restrict__ rgba_hq, uint64_t npx,
                               uint32_t background, int clear, uint32_t* __restrict__ status) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  bool overflow = false;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npx; i += stride) {
    const unsigned long long k = keys[i];
    const ulonglong2 a = accum[i];
    rgba_basic[i] = k == kEmptyKey ? background : ((uint32_t)(k & 0xFFFFFFu) | 0xFF000000u);
    const uint32_t c = (uint32_t)(a.y >> 32);
    uint32_t r, g, b;
    if (c == 0) {
      rgba_hq[i] = background;
    } else {
      if (c <= (1u << 24)) {  // as in k_resolve_hq: 32-bit quotients below the overflow bound
        const uint32_t h = c / 2;
        r = ((uint32_t)a.x + h) / c;
        g = ((uint32_t)(a.x >> 32) + h) / c;
        b = ((uint32_t)a.y + h) / c;
      } else {
        overflow = true;
        r = (uint32_t)(((a.x & 0xFFFFFFFFull) + c / 2) / c);
        g = (uint32_t)(((a.x >> 32) + c / 2) / c);
        b = (uint32_t)(((a.y & 0xFFFFFFFFull) + c / 2) / c);
      }
      rgba_hq[i] = (r & 0xFFu) | ((g & 0xFFu) << 8) | ((b & 0xFFu) << 16) | 0xFF000000u;
    }
    if (clear) {
      keys[i] = kEmptyKey;
      accum[i] = make_ulonglong2(0ull, 0ull);
    }
  }
  if (overflow) atomicOr(status, kStatusOverflow);
}

}  // namespace pcr
