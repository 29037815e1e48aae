// Roofline probes (include/pcr_ceilings.h): random u64 L2 atomics and 16-byte streaming reads.
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
