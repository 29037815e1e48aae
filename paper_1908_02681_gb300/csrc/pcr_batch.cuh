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
//   * one persistent launch per pass for all views: work items are (range of consecutive chunks, view),
//     taken range by range from a counter, so a range is read from HBM once for all views; a block
//     reloads a view's depth table when its view changes. The range size, points per thread, grid size and
//     same-pixel merging are launch tuning (BatchTuning), picked by an autotuner (pcr_batch_autotune).
//   * one resolve launch for all views.
#pragma once

#include "pcr_certified.cuh"

namespace pcr {

constexpr int kChunk = 1024;        // points per chunk (bounding box granularity)
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

constexpr int kMaxSliceWords = 4;  // largest work item: 4 mask words = 128 chunks

// Launch tuning of a batched frame (pcr_batch_tuning in include/pcr.h). Results never depend on it.
struct BatchTuning {
  int route = 0;              // 0: automatic (per-view passes for few views or large clouds), 1: batch kernel,
                              // 2: one single-view pass per view
  int slice_words = 1;        // mask words (32 chunks each) per work item: 1, 2 or 4
  int points_per_thread = 1;  // points a thread classifies per step: 1 or 2
  int blocks_per_sm = 4;      // capped at the blocks that can be resident
  int merge_width = 0;        // 0: one atomic per fragment; 8, 16 or 32: same-pixel fragments of that many
                              // lanes merged first
};

// Pass 1 (kHq = false) or pass 2 (kHq = true) for every view of a batch, one persistent launch. Work item
// = (range r of slice_words consecutive mask words, i.e. 32 * slice_words chunks, view v), numbered
// r * n_views + v and taken in that order from next_item[kHq]: the views of one range run close together in
// time, so the range's points come from HBM once and from L2 for the other views. Warp 0 lists the range's
// chunks whose mask bit is set; the block then walks them in steps of kCertThreads * kPts points (each warp
// takes 32 * kPts consecutive points per step), loading the next step's points before classifying the
// current ones. params: per-view CertParams in device memory (tier 2 and the FP64 arbiter read them there;
// tier 1 holds its constants in registers for the item). merge_width: see BatchTuning (kMerge = width > 0).
#ifndef PCR_BATCH_MIN_BLOCKS
#define PCR_BATCH_MIN_BLOCKS 4
#endif
template <bool kHq, bool kMerge, int kPts>
__global__ void __launch_bounds__(kCertThreads, PCR_BATCH_MIN_BLOCKS) k_batch_pass(
    const uint4* __restrict__ pts, uint64_t n, const CertParams* __restrict__ params,
    const BatchSlot* __restrict__ slots, const uint32_t* __restrict__ masks, uint32_t n_views, uint32_t n_chunks,
    uint32_t* __restrict__ next_item, uint32_t eps_num, uint32_t eps_den, uint32_t slice_words,
    uint32_t merge_width) {
  __shared__ long long sF[3 * kTableEntries];
  __shared__ uint4 queue[kCertWarps][kQueue];
  __shared__ uint32_t s_chunks[kMaxSliceWords * 32];
  __shared__ uint32_t s_item, s_nvis;
  static_assert(kPts == 1 || kPts == 2, "one or two points per thread per step");
  static_assert(kChunk % (kCertThreads * kPts) == 0, "whole steps per chunk");
  constexpr uint32_t kSteps = kChunk / (kCertThreads * kPts);  // steps per chunk
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint4* q = queue[warp];
  const uint32_t words = (n_chunks + 31u) / 32u;
  const uint32_t ranges = (words + slice_words - 1u) / slice_words;
  const uint32_t total = ranges * n_views;
  const uint32_t seg = merge_segment(lane, merge_width);
  uint32_t cur_view = 0xFFFFFFFFu;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next_item + (kHq ? 1 : 0), 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= total) break;
    const uint32_t r = item / n_views, v = item - r * n_views;
    const uint32_t w0 = r * slice_words;
    const uint32_t wn = words - w0 < slice_words ? words - w0 : slice_words;
    if (warp == 0) {  // the visible chunks of the item, in increasing order
      uint32_t cnt = 0;
      for (uint32_t k = 0; k < wn; ++k) {
        const uint32_t bits = masks[(uint64_t)v * words + w0 + k];
        if ((bits >> lane) & 1u) s_chunks[cnt + __popc(bits & ((1u << lane) - 1u))] = (w0 + k) * 32u + lane;
        cnt += __popc(bits);
      }
      if (lane == 0) s_nvis = cnt;
    }
    __syncthreads();
    const uint32_t nvis = s_nvis;
    if (nvis == 0u) continue;  // nothing of this range is visible in this view (the same in every thread)
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
    const uint32_t steps = nvis * kSteps;
    // first point of this warp in step st: chunk s_chunks[st / kSteps], part st % kSteps of it
    auto first = [&](uint32_t st) -> uint64_t {
      return (uint64_t)s_chunks[st / kSteps] * kChunk + (st % kSteps) * (kCertThreads * kPts) + warp * (32u * kPts) +
             lane;
    };
    auto load = [&](uint64_t i) { return i < n ? ld_stream16(pts + i) : make_uint4(0u, 0u, 0u, 0u); };
    // one point: tier 1, then the pass's commit, then the deferral of a point tier 1 could not decide
    auto point = [&](const uint4& p, bool valid) {
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
          defer = f.state >= kAmbiguous;  // undecided pixel, or code undecided between two neighbours: tier 2
        }
        commit_min<kMerge>(has && key < stored_key(keys, pix), pix, key, keys, lane, seg);
        unsigned dummy = 0;
        defer_points(defer, p, q, qn, lane, [&](const uint4& d) { raster_deferred(Pg, sF, d, keys, &dummy); });
      } else {
        bool accept = false;
        uint32_t pix = 0;
        if (valid) {
          const FastFrag f = classify_fast(H, sF, p);
          pix = f.pixel;
          defer = f.state >= kAmbiguous;
          if (f.state == kExact)
            accept = in_band(code_from_fixed(f.a1, f.a2), stored_key(keys, pix) >> 24, Pg.v.nq, eps_num, eps_den);
        }
        if constexpr (kMerge)
          commit_add<true>(accept, pix, p.w, accum, lane, seg);
        else  // consecutive points in adjacent lanes: merged in lane pairs (commit_add_pairs)
          commit_add_pairs(accept, pix, p.w, accum, lane);
        defer_points(defer, p, q, qn, lane,
                     [&](const uint4& d) { hq_deferred(Pg, sF, d, keys, accum, eps_num, eps_den); });
      }
    };
    uint64_t i_next = first(0);
    uint4 a0 = load(i_next), a1 = kPts == 2 ? load(i_next + 32) : a0;
#pragma unroll 1
    for (uint32_t st = 0; st < steps; ++st) {
      const uint64_t i = i_next;
      const uint4 c0 = a0, c1 = a1;
      if (st + 1 < steps) {  // the next step's points, requested before this step's are classified
        i_next = first(st + 1);
        a0 = load(i_next);
        if (kPts == 2) a1 = load(i_next + 32);
      }
      point(c0, i < n);
      if (kPts == 2) point(c1, i + 32 < n);
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

// Launches the batch pass kernel of a tuning (template instance by merging and points per thread).
template <bool kHq>
inline void batch_pass_launch(const BatchTuning& t, int sms, int resident, const uint4* pts, uint64_t n,
                              const CertParams* params, const BatchSlot* slots, const uint32_t* masks,
                              uint32_t n_views, uint32_t n_chunks, uint32_t* next_item, uint32_t eps_num,
                              uint32_t eps_den, cudaStream_t s) {
  const int per_sm = t.blocks_per_sm < resident ? t.blocks_per_sm : resident;
  const unsigned grid = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
  const uint32_t sw = (uint32_t)t.slice_words, mw = (uint32_t)t.merge_width;
#define PCR_BATCH_LAUNCH(M, K)                                                                                    \
  k_batch_pass<kHq, M, K><<<grid, kCertThreads, 0, s>>>(pts, n, params, slots, masks, n_views, n_chunks, next_item, \
                                                        eps_num, eps_den, sw, mw)
  if (t.merge_width > 0) {
    if (t.points_per_thread == 2) PCR_BATCH_LAUNCH(true, 2); else PCR_BATCH_LAUNCH(true, 1);
  } else {
    if (t.points_per_thread == 2) PCR_BATCH_LAUNCH(false, 2); else PCR_BATCH_LAUNCH(false, 1);
  }
#undef PCR_BATCH_LAUNCH
}

// Resident blocks per SM of the batch pass kernel of a tuning.
template <bool kHq>
inline int batch_pass_resident(const BatchTuning& t) {
  int b = 0;
  cudaError_t e;
  if (t.merge_width > 0)
    e = t.points_per_thread == 2
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_pass<kHq, true, 2>, kCertThreads, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_pass<kHq, true, 1>, kCertThreads, 0);
  else
    e = t.points_per_thread == 2
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_pass<kHq, false, 2>, kCertThreads, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_pass<kHq, false, 1>, kCertThreads, 0);
  if (e != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 1;
  }
  return b;
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
