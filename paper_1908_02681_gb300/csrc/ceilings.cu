// Roofline probes (include/pcr_ceilings.h): random u64 L2 atomics, 16-byte streaming reads, the passes'
// framebuffer operations replayed without the transform, and the FP64 / FP32 fused multiply-add rates.
#include <cstdint>
#include <cuda_runtime.h>

#include "pcr_ceilings.h"
#include "pcr_device.cuh"

namespace {

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

__global__ void __launch_bounds__(512) k_random_atomics(unsigned long long* slots, uint32_t n_slots, uint64_t n_ops,
                                                        int op) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_ops; i += stride) {
    const uint32_t h = mix32((uint32_t)i ^ (uint32_t)(i >> 32) * 0x9E3779B9u);
    const uint32_t idx = (uint32_t)(((uint64_t)h * n_slots) >> 32);
    if (op == 0)
      atomicMin(slots + idx, ((unsigned long long)mix32(h) << 24) | (i & 0xFFFFFF));
    else
      atomicAdd(slots + idx, (unsigned long long)(i & 0xFF) | (1ull << 32));
  }
}

__global__ void __launch_bounds__(256) k_stream_read(const uint4* __restrict__ src, uint64_t n, uint32_t* sink) {
  uint32_t acc = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 v = pcr::ld_stream16(src + i);
    acc ^= v.x + v.y + v.z + v.w;
  }
  if (acc == 0x9E3779B9u) sink[(uint64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// The visible fragments of a view in the order of the points: pixel (0xFFFFFFFF when culled) and key, by
// the FP64 definition with linear depth. Run once, outside any timed region.
__global__ void __launch_bounds__(256) k_pattern_project(const uint4* __restrict__ pts, uint64_t n, const pcr::DevView v,
                                                         uint32_t* __restrict__ pix, unsigned long long* __restrict__ key) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 p = pts[i];
    uint32_t px;
    unsigned long long q;
    const bool vis = pcr::project_fp64(v, __uint_as_float(p.x), __uint_as_float(p.y), __uint_as_float(p.z), &px, &q);
    pix[i] = vis ? px : 0xFFFFFFFFu;
    key[i] = vis ? pcr::make_key(q, p.w) : pcr::kEmptyKey;
  }
}

// Pass 1 without the transform: one atomic minimum per visible fragment, in the order of the points (a warp
// takes 32 consecutive points per step, as the passes do). Reads 12 B per point. With `filter`, each fragment
// first reads the stored key (from L2) and skips the atomic unless its key is smaller: the stored key only
// decreases, so a skipped key could never have become the minimum.
__global__ void __launch_bounds__(256) k_pattern_min(const uint32_t* __restrict__ pix,
                                                     const unsigned long long* __restrict__ key, uint64_t n,
                                                     unsigned long long* __restrict__ keys, int filter) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t p = __ldcs(pix + i);
    const unsigned long long k = __ldcs(key + i);
    if (p != 0xFFFFFFFFu && (!filter || k < __ldcg(keys + p))) atomicMin(keys + p, k);
  }
}

// Pass 2 without the transform: per visible fragment the stored key of its pixel, the band test, and for an
// accepted fragment the two colour/count additions.
__global__ void __launch_bounds__(256) k_pattern_hq(const uint32_t* __restrict__ pix,
                                                    const unsigned long long* __restrict__ key, uint64_t n,
                                                    const unsigned long long* __restrict__ keys,
                                                    unsigned long long* __restrict__ accum, uint32_t eps_num,
                                                    uint32_t eps_den, unsigned long long nq) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t p = __ldcs(pix + i);
    const unsigned long long k = __ldcs(key + i);
    if (p == 0xFFFFFFFFu) continue;
    if (pcr::in_band(k >> 24, keys[p] >> 24, nq, eps_num, eps_den)) {
      atomicAdd(accum + 2 * (uint64_t)p, pcr::hq_rg((uint32_t)k));
      atomicAdd(accum + 2 * (uint64_t)p + 1, pcr::hq_bc((uint32_t)k));
    }
  }
}

// Fused multiply-add throughput: every thread runs kFmaChains independent chains of `iters` fmas each
// (explicitly rounded, so nothing is contracted or folded), then writes to sink only when the sum hits an
// impossible value. The chains hide the pipe latency at full occupancy.
constexpr int kFmaChains = 16;
constexpr int kFmaThreads = 256;
constexpr int kFmaBlocksPerSm = 8;

__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(kFmaThreads) k_fma(uint32_t iters, uint32_t* sink) {
  T a[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) a[k] = (T)(threadIdx.x + 1 + k) * (T)0.001;
  const T b = (T)0.9999, c = (T)0.0001;
#pragma unroll 1
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = fma_rn(a[k], b, c);
  }
  T s = (T)0;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += a[k];
  if (s == (T)-1.0) sink[(uint64_t)blockIdx.x * blockDim.x + threadIdx.x] = 1u;
}

int sms() {
  int dev = 0, v = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

}  // namespace

extern "C" int pcr_ceiling_random_atomics(uint64_t* d_slots, uint32_t n_slots, uint64_t n_ops, int32_t op,
                                          void* stream) {
  if (!d_slots || n_slots == 0 || n_ops >= (1ull << 40) || (op != 0 && op != 1)) return (int)cudaErrorInvalidValue;
  if (n_ops == 0) return 0;
  k_random_atomics<<<sms() * 4, 512, 0, (cudaStream_t)stream>>>(reinterpret_cast<unsigned long long*>(d_slots),
                                                                 n_slots, n_ops, op);
  return (int)cudaGetLastError();
}

extern "C" int pcr_ceiling_stream_read(const void* d_src, uint64_t n16, uint32_t* d_sink, void* stream) {
  if (!d_src || !d_sink || (reinterpret_cast<uintptr_t>(d_src) & 15u)) return (int)cudaErrorInvalidValue;
  if (n16 == 0) return 0;
  k_stream_read<<<sms() * 64, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const uint4*>(d_src), n16, d_sink);
  return (int)cudaGetLastError();
}

extern "C" int pcr_ceiling_pattern_project(const void* d_points, uint64_t n, const double* m12, double near_,
                                           double far_, int32_t width, int32_t height, uint32_t* d_pix,
                                           uint64_t* d_key, void* stream) {
  if (!d_points || !m12 || !d_pix || !d_key || width < 1 || height < 1 || width > 16384 || height > 16384 ||
      !(near_ > 0.0) || !(far_ > near_) || (reinterpret_cast<uintptr_t>(d_points) & 15u))
    return (int)cudaErrorInvalidValue;
  if (n == 0) return 0;
  pcr::DevView v{};
  for (int i = 0; i < 12; ++i) v.m[i] = m12[i];
  v.near_ = near_;
  v.far_ = far_;
  v.scale = 1099511627776.0 / (far_ - near_);
  v.fwidth = (float)width;
  v.fheight = (float)height;
  v.width = width;
  v.height = height;
  v.depth_mode = 0;
  k_pattern_project<<<sms() * 8, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const uint4*>(d_points), n, v,
                                                                  d_pix, reinterpret_cast<unsigned long long*>(d_key));
  return (int)cudaGetLastError();
}

extern "C" int pcr_ceiling_pattern_min(const uint32_t* d_pix, const uint64_t* d_key, uint64_t n, uint64_t* d_keys,
                                       int32_t filter, void* stream) {
  if (!d_pix || !d_key || !d_keys || (filter != 0 && filter != 1)) return (int)cudaErrorInvalidValue;
  if (n == 0) return 0;
  k_pattern_min<<<sms() * 8, 256, 0, (cudaStream_t)stream>>>(
      d_pix, reinterpret_cast<const unsigned long long*>(d_key), n, reinterpret_cast<unsigned long long*>(d_keys),
      filter);
  return (int)cudaGetLastError();
}

extern "C" int pcr_ceiling_pattern_hq(const uint32_t* d_pix, const uint64_t* d_key, uint64_t n, const uint64_t* d_keys,
                                      uint64_t* d_accum, uint32_t eps_num, uint32_t eps_den, uint64_t nq,
                                      void* stream) {
  if (!d_pix || !d_key || !d_keys || !d_accum || eps_den == 0) return (int)cudaErrorInvalidValue;
  if (n == 0) return 0;
  k_pattern_hq<<<sms() * 8, 256, 0, (cudaStream_t)stream>>>(
      d_pix, reinterpret_cast<const unsigned long long*>(d_key), n,
      reinterpret_cast<const unsigned long long*>(d_keys), reinterpret_cast<unsigned long long*>(d_accum), eps_num,
      eps_den, nq);
  return (int)cudaGetLastError();
}

extern "C" int pcr_ceiling_fma(int32_t fp64, uint32_t iters, uint32_t* d_sink, uint64_t* fmas, void* stream) {
  if (!d_sink || !fmas || (fp64 != 0 && fp64 != 1) || iters == 0) return (int)cudaErrorInvalidValue;
  const unsigned grid = (unsigned)(sms() * kFmaBlocksPerSm);
  *fmas = (uint64_t)grid * kFmaThreads * kFmaChains * iters;
  if (fp64)
    k_fma<double><<<grid, kFmaThreads, 0, (cudaStream_t)stream>>>(iters, d_sink);
  else
    k_fma<float><<<grid, kFmaThreads, 0, (cudaStream_t)stream>>>(iters, d_sink);
  return (int)cudaGetLastError();
}
