// Batched rendering of a resident point cloud: many views per persistent launch.
//
// The per-point work is the certified transform of pcr_certified.cuh (Sections 2.1 and 2.2 of arXiv
// 1908.02681, same results bit for bit). What batching adds:
//   * chunk culling: the cloud is cut into chunks of kChunk consecutive points whose bounding boxes are
//     computed once (k_chunk_bounds). Per view, a chunk is skipped when every point of its box is culled
//     by the definition: the affine functions w - near, far - w, (1 + 1e-5) w -+ cx, (1 + 1e-5) w -+ cy
//     reach their maximum over a box at a corner, and when that maximum, evaluated in float, stays below
//     zero by more than a rounding bound (16u times the magnitude sum), every point of the box is behind
//     the near plane, beyond the far plane, or at |ndc| > 1 + 1e-5, which the definition's float pixel
//     mapping (relative error below 1e-6) sends outside the image. A box with a NaN or infinite bound is
//     never skipped.
//   * one persistent launch per pass for all views: work items are (range of kSlice consecutive chunks,
//     view), taken range by range from a counter, so a range is read from HBM once for all views; a block
//     reloads a view's depth table when its view changes.
//   * one resolve launch for all views.
#pragma once

#include "pcr_certified.cuh"

namespace pcr {

constexpr int kChunk = 1024;        // points per chunk (bounding box granularity)
constexpr int kSlice = 32;          // consecutive chunks per work item (one word of a view's mask)
constexpr int kMaxBatchViews = 256;

// Per-view constants of a batch that live in device memory (read once per work item).
struct BatchSlot {
  unsigned long long* keys;
  unsigned long long* accum;  // HQ framebuffers, else null
  uint32_t* out;              // resolve output (pcr_resolve_batch), else null
  uint32_t* status;
  int32_t width, height;
  int32_t hq;
  int32_t pad;
  // chunk culling planes: value = a . (x, y, z) + b; a chunk is culled when one plane's maximum over the
  // box plus its rounding margin is negative
  float plane_a[6][3];
  float plane_b[6];
};

// ------------------------------------------------------------------------------------------------ cloud

// Bounding box of every chunk: lo.xyz, hi.xyz (6 floats). A chunk holding a non-finite coordinate gets
// NaN bounds (never culled).
__global__ void __launch_bounds__(256) k_chunk_bounds(const uint4* __restrict__ pts, uint64_t n, float* __restrict__ bounds,
                                                      uint64_t n_chunks) {
  __shared__ float red[6][8];
  __shared__ int bad_s;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (uint64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    int bad = 0;
    const uint64_t b = c * kChunk;
    for (uint32_t k = threadIdx.x; k < (uint32_t)kChunk; k += blockDim.x) {
      const uint64_t i = b + k;
      if (i >= n) break;
      const uint4 p = ld_stream16(pts + i);
      const float v[3] = {__uint_as_float(p.x), __uint_as_float(p.y), __uint_as_float(p.z)};
      for (int j = 0; j < 3; ++j) {
        bad |= !(fabsf(v[j]) <= 3.0e38f);
        lo[j] = fminf(lo[j], v[j]);
        hi[j] = fmaxf(hi[j], v[j]);
      }
    }
    for (int j = 0; j < 3; ++j) {
      for (int o = 16; o > 0; o >>= 1) {
        lo[j] = fminf(lo[j], __shfl_xor_sync(0xFFFFFFFFu, lo[j], o));
        hi[j] = fmaxf(hi[j], __shfl_xor_sync(0xFFFFFFFFu, hi[j], o));
      }
    }
    bad = __any_sync(0xFFFFFFFFu, bad);
    if (threadIdx.x == 0) bad_s = 0;
    __syncthreads();
    if (lane == 0) {
      for (int j = 0; j < 3; ++j) {
        red[j][warp] = lo[j];
        red[3 + j][warp] = hi[j];
      }
      if (bad) atomicOr(&bad_s, 1);
    }
    __syncthreads();
    if (threadIdx.x < 6) {
      float r = red[threadIdx.x][0];
      for (uint32_t w = 1; w < blockDim.x / 32; ++w)
        r = threadIdx.x < 3 ? fminf(r, red[threadIdx.x][w]) : fmaxf(r, red[threadIdx.x][w]);
      bounds[c * 6 + threadIdx.x] = bad_s ? __int_as_float(0x7FC00000) : r;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------------------------- culling

// For each (view, chunk): bit c of the view's visibility mask is set unless chunk c's box is certainly
// culled. Thread per chunk, one 32-bit mask word per warp (a ballot, no atomics); the grid's y dimension
// is the view. counts[v] (zeroed before) receives the number of visible chunks.
__global__ void __launch_bounds__(256) k_cull(const float* __restrict__ bounds, uint32_t n_chunks,
                                              const BatchSlot* __restrict__ slots, uint32_t* __restrict__ masks,
                                              uint32_t* __restrict__ counts) {
  const uint32_t v = blockIdx.y;
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  bool keep = false;
  if (c < n_chunks) {
    const float* bb = bounds + (uint64_t)c * 6;
    const float lo[3] = {bb[0], bb[1], bb[2]}, hi[3] = {bb[3], bb[4], bb[5]};
    const BatchSlot& S = slots[v];
    bool culled = false;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float mx = S.plane_b[k], mag = fabsf(S.plane_b[k]);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float a = S.plane_a[k][j];
        const float t0 = __fmul_rn(a, lo[j]), t1 = __fmul_rn(a, hi[j]);
        mx = __fadd_rn(mx, fmaxf(t0, t1));
        mag = __fadd_rn(mag, fmaxf(fabsf(t0), fabsf(t1)));
      }
      // every rounding of the float evaluation and of the coefficients stays below 16u * mag
      culled |= __fmaf_rn(16.0f * 0x1p-24f, mag, mx) < 0.0f;
    }
    keep = !culled;  // NaN bounds: every comparison false, never culled
  }
  const unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
  const uint32_t words = (n_chunks + 31u) / 32u;
  if ((threadIdx.x & 31u) == 0u && c / 32u < words) {
    masks[(uint64_t)v * words + c / 32u] = m;
    if (m) atomicAdd(counts + v, (uint32_t)__popc(m));
  }
}

// Resets the two work-item counters (pass 1, pass 2) of a frame.
__global__ void k_items(uint32_t* __restrict__ next_item) {
  if (threadIdx.x < 2) next_item[threadIdx.x] = 0u;
}

// ------------------------------------------------------------------------------------------- batch passes

// Pass 1 (kHq = false) or pass 2 (kHq = true) for every view of a batch, one persistent launch. Work item
// = (range r of kSlice consecutive chunks, view v), numbered r * n_views + v and taken in that order from
// next_item[kHq]: the views of one range run close together in time, so the range's points come from HBM
// once and from L2 for the other views. An item covers the range's chunks whose mask bit is set.
// params: per-view CertParams in device memory (tier 2 and the FP64 arbiter read them there; tier 1 holds
// its constants in registers for the item).
template <bool kHq>
#ifndef PCR_BATCH_MIN_BLOCKS
#define PCR_BATCH_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(kCertThreads, PCR_BATCH_MIN_BLOCKS) k_batch_pass(const uint4* __restrict__ pts, uint64_t n,
                                                             const CertParams* __restrict__ params,
                                                             const BatchSlot* __restrict__ slots,
                                                             const uint32_t* __restrict__ masks, uint32_t n_views,
                                                             uint32_t n_chunks, uint32_t* __restrict__ next_item,
                                                             uint32_t eps_num, uint32_t eps_den) {
  __shared__ long long sF[3 * kTableEntries];
  __shared__ uint4 queue[kCertWarps][kQueue];
  __shared__ uint32_t s_item;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint4* q = queue[warp];
  static_assert(kSlice == 32, "a range is one word of the view's mask");
  const uint32_t words = (n_chunks + 31u) / 32u;
  const uint32_t total = (n_chunks + kSlice - 1) / kSlice * n_views;
  uint32_t cur_view = 0xFFFFFFFFu;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next_item + (kHq ? 1 : 0), 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= total) break;
    const uint32_t r = item / n_views, v = item - r * n_views;
    const uint32_t c0 = r * kSlice;
    const uint32_t bits = masks[(uint64_t)v * words + c0 / 32u];  // kSlice == 32: the whole word
    if (bits == 0u) {  // nothing of this range is visible in this view (the same in every thread)
      __syncthreads();
      continue;
    }
    if (v != cur_view) {
      const long long* src = &params[v].F[0][0];
      for (int i = threadIdx.x; i < 3 * kTableEntries; i += blockDim.x) sF[i] = src[i];
      cur_view = v;
    }
    __syncthreads();
    const CertParams& Pg = params[v];
    const HotParams H = hot_params(Pg);
    const BatchSlot& S = slots[v];
    unsigned long long* const keys = S.keys;
    unsigned long long* const accum = S.accum;
    // the framebuffer pointers come from device memory, so the compiler cannot infer their address space;
    // stated here, the atomics compile to fire-and-forget global reductions instead of generic atomics that
    // return the old value
    __builtin_assume(__isGlobal(keys));
    __builtin_assume(accum == nullptr || __isGlobal(accum));
    uint32_t qn = 0;
    // the item's points as one sequence of steps (kChunk / kCertThreads per chunk); the point of the next
    // step is loaded before the current one is classified, so its memory latency overlaps the work
    static_assert(kChunk % kCertThreads == 0, "whole steps per chunk");
    constexpr uint32_t kPerChunk = kChunk / kCertThreads;
    const uint32_t steps = (uint32_t)__popc(bits) * kPerChunk;
    // the chunk of the next step and its part: visible chunks in increasing order (lowest remaining bit)
    uint32_t rem = bits & (bits - 1u), nc = c0 + (uint32_t)(__ffs(bits) - 1), nk = 0;
    uint64_t i_next = (uint64_t)nc * kChunk + warp * 32u + lane;
    uint4 p_next = i_next < n ? ld_stream16(pts + i_next) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 1
    for (uint32_t st = 0; st < steps; ++st) {
      {
        const uint64_t i = i_next;
        const bool valid = i < n;
        const uint4 p = p_next;
        if (st + 1 < steps) {
          if (++nk == kPerChunk) {  // next visible chunk of the range (there is one: more steps remain)
            nk = 0;
            nc = c0 + (uint32_t)(__ffs(rem) - 1);
            rem &= rem - 1u;
          }
          i_next = (uint64_t)nc * kChunk + nk * kCertThreads + warp * 32u + lane;
          p_next = i_next < n ? ld_stream16(pts + i_next) : make_uint4(0u, 0u, 0u, 0u);
        }
        bool defer = false;
        if (!kHq) {
          bool has = false;
          uint32_t pix = 0;
          unsigned long long key = 0;
          if (valid) {
            const FastFrag f = classify_fast(H, sF, p);
            pix = f.pixel;
            key = key_from_fixed(f.a0, f.a1, f.a2, p.w);
            has = f.state == kExact;
            defer = f.state == kDefer;
            if (f.state == kAmbiguous) {
              const unsigned long long klo = f.lo_half ? key - (1ull << 24) : key;
              defer = klo < keys[pix];
            }
          }
          if (has && key < stored_key(keys, pix)) atomicMin(keys + pix, key);
          unsigned dummy = 0;
          defer_points(defer, p, q, qn, lane, [&](const uint4& d) { raster_deferred(Pg, sF, d, keys, &dummy); });
        } else {
          bool accept = false;
          uint32_t pix = 0;
          if (valid) {
            const FastFrag f = classify_fast(H, sF, p);
            pix = f.pixel;
            defer = f.state == kDefer;
            if (f.state == kExact || f.state == kAmbiguous) {
              const unsigned long long qmin = keys[pix] >> 24;
              const unsigned long long qc = code_from_fixed(f.a1, f.a2);
              bool acc = in_band(f.state == kAmbiguous && f.lo_half ? qc - 1 : qc, qmin, Pg.v.nq, eps_num, eps_den);
              if (f.state == kAmbiguous) {
                const bool other = in_band(f.lo_half ? qc : qc + 1, qmin, Pg.v.nq, eps_num, eps_den);
                defer = acc != other;
                acc = acc && !defer;
              }
              accept = acc;
            }
          }
          if (accept) hq_add(accum, pix, p.w);
          defer_points(defer, p, q, qn, lane,
                       [&](const uint4& d) { hq_deferred(Pg, sF, d, keys, accum, eps_num, eps_den); });
        }
      }
    }
    // the queue holds points of this view only: finish them before the next item
    if (lane < qn) {
      if (!kHq) {
        unsigned dummy = 0;
        raster_deferred(Pg, sF, q[lane], keys, &dummy);
      } else {
        hq_deferred(Pg, sF, q[lane], keys, accum, eps_num, eps_den);
      }
    }
    __syncwarp();
    __syncthreads();
  }
}

// Resolve of every framebuffer of a batch (pcr_resolve semantics per view), one launch. pixel_start[v] =
// first global pixel of view v, pixel_start[n_views] = total.
__global__ void __launch_bounds__(256) k_resolve_batch(const BatchSlot* __restrict__ slots,
                                                       const uint64_t* __restrict__ pixel_start, uint32_t n_views,
                                                       uint32_t background, int clear) {
  const uint64_t total = pixel_start[n_views];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    uint32_t v = 0;
    uint32_t lo = 0, hi = n_views;  // last v with pixel_start[v] <= g
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (pixel_start[mid] <= g) lo = mid; else hi = mid;
    }
    v = lo;
    const BatchSlot& S = slots[v];
    const uint64_t i = g - pixel_start[v];
    unsigned long long* keys = S.keys;
    ulonglong2* acc = reinterpret_cast<ulonglong2*>(S.accum);
    if (S.hq) {
      const ulonglong2 a = acc[i];
      const uint32_t c = (uint32_t)(a.y >> 32);
      if (c == 0) {
        S.out[i] = background;
      } else {
        if (c > (1u << 24)) atomicOr(S.status, kStatusOverflow);
        const uint32_t r = (uint32_t)(((a.x & 0xFFFFFFFFull) + c / 2) / c);
        const uint32_t gg = (uint32_t)(((a.x >> 32) + c / 2) / c);
        const uint32_t b = (uint32_t)(((a.y & 0xFFFFFFFFull) + c / 2) / c);
        S.out[i] = (r & 0xFFu) | ((gg & 0xFFu) << 8) | ((b & 0xFFu) << 16) | 0xFF000000u;
      }
      if (clear) {
        acc[i] = make_ulonglong2(0ull, 0ull);
        keys[i] = kEmptyKey;
      }
    } else {
      const unsigned long long k = keys[i];
      S.out[i] = k == kEmptyKey ? background : ((uint32_t)(k & 0xFFFFFFu) | 0xFF000000u);
      if (clear) {
        keys[i] = kEmptyKey;
        if (acc) acc[i] = make_ulonglong2(0ull, 0ull);
      }
    }
  }
}

}  // namespace pcr
