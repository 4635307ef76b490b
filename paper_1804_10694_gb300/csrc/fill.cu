// Timing inputs for the tuner: uniform[-1, 1) values from a counter-based
// hash of (seed, index) (SplitMix64 finaliser), so that tuning runs on
// realistic, non-zero data without any host-to-device traffic.
#include <cuda_runtime.h>

#include <cstdint>

#include "runtime.h"

namespace gb {
namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void fill_uniform_kernel(float* __restrict__ x, size_t n, uint64_t seed) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const uint64_t h = splitmix64(seed * 0x632BE59BD9B4E019ull + i);
    // 24 random bits -> [0, 1) exactly representable, then to [-1, 1)
    const float u = static_cast<float>(h >> 40) * (1.0f / 16777216.0f);
    x[i] = 2.0f * u - 1.0f;
  }
}

}  // namespace

cudaError_t fill_uniform_launch(float* x, size_t n, uint64_t seed, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  fill_uniform_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(x, n, seed);
  return cudaGetLastError();
}

}  // namespace gb
