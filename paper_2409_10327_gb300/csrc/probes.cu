// Roofline probes: the two rates the renderer's kernels are compared with
// that neither a stream copy nor a library GEMM measures.
//
//  * Random gathers from an L2-resident table.  The secondary hash encode
//    reads 4- or 8-byte table entries at scattered rows of a 32-64 MB table
//    that stays in the 129 MB L2, so its ceiling is the rate at which the
//    SMs can have such loads served, not HBM bandwidth.  The probe runs the
//    same access pattern with nothing else: every thread issues independent
//    loads at hashed rows of a table of the caller's size, 8 in flight.
//  * FP32 FMA throughput, for the FP32 kernels: 8 independent FMA chains per
//    thread, all SMs full.
//
// Both write one value per thread to `sink` so the work cannot be removed.
#include <cuda_fp16.h>

#include "rt_internal.h"

namespace rtk {

namespace {

// A 32-bit integer hash (a multiply-xorshift mix) of (thread, iteration): a
// row index uniform over the table, cheap next to a load.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

template <typename T>
__global__ void __launch_bounds__(512) gather_probe_kernel(const T* __restrict__ table, uint32_t mask,
                                                           int iters, uint32_t seed, uint32_t* __restrict__ sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  uint32_t base = mix32(tid ^ seed);
  for (int it = 0; it < iters; ++it) {
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __ldg(table + (mix32(base + (uint32_t)(8 * it + k)) & mask));
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if constexpr (sizeof(T) == 8) {
        acc ^= v[k].x ^ v[k].y;
      } else {
        acc ^= v[k];
      }
    }
  }
  sink[tid] = acc;
}

__global__ void __launch_bounds__(512) ffma_probe_kernel(int iters, float seed, float* __restrict__ sink) {
  const float b = 1.0f + 1e-7f * (float)(threadIdx.x & 7);
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + (float)k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, -1e-7f);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

}  // namespace rtk

using namespace rtk;

extern "C" rt_status rt_probe_gather(const void* table, int64_t rows, int32_t bytes_per_load, int32_t iters,
                                     int32_t blocks, uint32_t* sink, void* stream) {
  if (table == nullptr || sink == nullptr || rows < 2 || (rows & (rows - 1)) != 0 || rows > (1LL << 31) ||
      (bytes_per_load != 4 && bytes_per_load != 8) || iters < 1 || blocks < 1 || blocks > 65535 ||
      (reinterpret_cast<uintptr_t>(table) % (uintptr_t)bytes_per_load) != 0 ||
      (reinterpret_cast<uintptr_t>(sink) % 4) != 0)
    return RT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t mask = (uint32_t)(rows - 1);
  if (bytes_per_load == 4)
    gather_probe_kernel<uint32_t><<<blocks, 512, 0, s>>>(static_cast<const uint32_t*>(table), mask, iters, 12345u,
                                                         sink);
  else
    gather_probe_kernel<uint2><<<blocks, 512, 0, s>>>(static_cast<const uint2*>(table), mask, iters, 12345u, sink);
  return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}

extern "C" rt_status rt_probe_ffma(int32_t iters, int32_t blocks, float* sink, void* stream) {
  if (sink == nullptr || iters < 1 || blocks < 1 || blocks > 65535 || (reinterpret_cast<uintptr_t>(sink) % 4) != 0)
    return RT_ERR_INVALID_ARG;
  ffma_probe_kernel<<<blocks, 512, 0, static_cast<cudaStream_t>(stream)>>>(iters, 0.5f, sink);
  return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}
