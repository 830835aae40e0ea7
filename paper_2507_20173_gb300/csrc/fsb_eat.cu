// fsb_eat.cu -- the paper's eat() reduction on its own, with a choice of
// reduction construct: the GPU analogue of its Experiment 3 (Sec. 2.3.2,
// Sec. 3.4), which times eat() -- max over the school of
// (prevObjective - currentObjective) -- under OpenMP `reduction(max:)` and
// under a `critical` section.
//
// Constructs (all exact: max is order-free, taken on order-preserving keys):
//   kEatHierarchical  warp shuffle -> shared memory -> one atomicMax per
//                     block (the analogue of `reduction(max:)`)
//   kEatPerWarp       one atomicMax per warp
//   kEatPerFish       one atomicMax per fish on a single word (the analogue
//                     of `critical`: every update serialises on one address)
// The input is streamed once (8 B per fish in binary32); the result goes to
// a device word, decoded to binary64 on the host.
#include <cstdint>

#include "fsb_device.cuh"
#include "fsb_internal.h"
#include "fsb_reduce.cuh"

namespace fsb {
namespace {

__global__ void eat_key_reset(unsigned* key) { *key = 0u; }

// The winning order key back to the value max(prev - cur), as binary64.
__global__ void eat_key_decode(const unsigned* key, double* out) {
  *out = static_cast<double>(key_to_value(*key, 0.f));
}

template <int CONSTRUCT>
__global__ void __launch_bounds__(256) eat_max_kernel(const float* __restrict__ prev,
                                                      const float* __restrict__ cur, uint64_t n,
                                                      unsigned* key) {
  __shared__ unsigned s_key[8];
  unsigned best = 0u;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  const uint64_t n4 = n / 4;
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (uint64_t g = tid; g < n4; g += stride) {
    const float4 p = reinterpret_cast<const float4*>(prev)[g];
    const float4 c = reinterpret_cast<const float4*>(cur)[g];
    const unsigned k0 = order_key(__fsub_rn(p.x, c.x)), k1 = order_key(__fsub_rn(p.y, c.y));
    const unsigned k2 = order_key(__fsub_rn(p.z, c.z)), k3 = order_key(__fsub_rn(p.w, c.w));
    if (CONSTRUCT == kEatPerFish) {
      atomicMax(key, k0);
      atomicMax(key, k1);
      atomicMax(key, k2);
      atomicMax(key, k3);
    } else {
      best = max(best, max(max(k0, k1), max(k2, k3)));
    }
  }
  const uint64_t i = n4 * 4 + tid;  // ragged tail
  if (i < n) {
    const unsigned k = order_key(__fsub_rn(prev[i], cur[i]));
    if (CONSTRUCT == kEatPerFish)
      atomicMax(key, k);
    else
      best = max(best, k);
  }
  if (CONSTRUCT == kEatPerFish) return;
  best = warp_max(best);
  if (CONSTRUCT == kEatPerWarp) {
    if ((threadIdx.x & 31) == 0) atomicMax(key, best);
    return;
  }
  if ((threadIdx.x & 31) == 0) s_key[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < (blockDim.x >> 5) ? s_key[threadIdx.x] : 0u;
    best = warp_max(best);
    if (threadIdx.x == 0) atomicMax(key, best);
  }
}

}  // namespace

cudaError_t launch_eat_max(const float* prev, const float* cur, uint64_t n, int construct,
                           unsigned* key, double* value, int grid, cudaStream_t s) {
  eat_key_reset<<<1, 1, 0, s>>>(key);
  switch (construct) {
    case kEatHierarchical:
      eat_max_kernel<kEatHierarchical><<<grid, 256, 0, s>>>(prev, cur, n, key);
      break;
    case kEatPerWarp:
      eat_max_kernel<kEatPerWarp><<<grid, 256, 0, s>>>(prev, cur, n, key);
      break;
    case kEatPerFish:
      eat_max_kernel<kEatPerFish><<<grid, 256, 0, s>>>(prev, cur, n, key);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  eat_key_decode<<<1, 1, 0, s>>>(key, value);
  return cudaGetLastError();
}

}  // namespace fsb
