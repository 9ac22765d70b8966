// Measurement utility: the L2 random-gather ceiling that bounds the hash-table
// gather when the table is L2-resident (every lookup of a hashed level lands
// on an unrelated 32-byte sector).
#pragma once
#include "nbvh_internal.cuh"

namespace nbvh {

__device__ __forceinline__ uint32_t probe_mix(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

// kProbeLoads independent 4-byte loads per thread per iteration at positions
// masked to the table (n_entries a power of two), summed so none is dropped.
constexpr int kProbeLoads = 16;
static __global__ void __launch_bounds__(1024) probe_gather_kernel(const uint32_t* __restrict__ tab, uint32_t mask,
                                                            int iters, uint32_t* __restrict__ sink) {
  uint32_t s = probe_mix(blockIdx.x * blockDim.x + threadIdx.x + 12345u);
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
    uint32_t v[kProbeLoads];
#pragma unroll
    for (int u = 0; u < kProbeLoads; ++u) v[u] = __ldg(tab + (probe_mix(s + u * 0x9e3779b9u) & mask));
#pragma unroll
    for (int u = 0; u < kProbeLoads; ++u) acc += v[u];
    s = probe_mix(s ^ acc);
  }
  if (acc == 0x9e3779b9u) sink[0] = acc;  // keeps the loads; practically never stores
}

// kProbeLoads fire-and-forget float2 atomic adds per thread per iteration at
// pseudo-random entries (n_entries a power of two): the form of the training
// backward's table-gradient updates at F = 2.
static __global__ void __launch_bounds__(1024) probe_reduce_kernel(float2* __restrict__ grad, uint32_t mask,
                                                                   int iters) {
  uint32_t s = probe_mix(blockIdx.x * blockDim.x + threadIdx.x + 777u);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kProbeLoads; ++u) {
      const uint32_t h = probe_mix(s + u * 0x9e3779b9u);
      atomicAdd(grad + (h & mask), make_float2(1e-30f, 1e-30f));
    }
    s = probe_mix(s + 0x85ebca6bu);
  }
}

}  // namespace nbvh
