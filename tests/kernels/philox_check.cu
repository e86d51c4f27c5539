// Cross-check of the library's device Philox4x32-10 (csrc/common.cuh) with
// the independent implementation in cuRAND's device header
// (curand_Philox4x32_10, counter and key as given), on pseudo-random
// counters and keys; compiled by tests/test_gpu_philox.py into a temporary
// shared library.
#include <curand_kernel.h>

#include "common.cuh"

namespace {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void philox_check_kernel(unsigned long long n, unsigned long long seed, unsigned long long *bad) {
  unsigned long long local = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long a = splitmix64(seed ^ (3 * i)), b = splitmix64(seed ^ (3 * i + 1)),
                             c = splitmix64(seed ^ (3 * i + 2));
    const uint32_t c0 = (uint32_t)a, c1 = (uint32_t)(a >> 32), c2 = (uint32_t)b, c3 = (uint32_t)(b >> 32);
    const uint32_t k0 = (uint32_t)c, k1 = (uint32_t)(c >> 32);
    const uint4 r = curand_Philox4x32_10(make_uint4(c0, c1, c2, c3), make_uint2(k0, k1));
    const trsgd::Philox4 o = trsgd::philox4x32_10(c0, c1, c2, c3, k0, k1);
    local += (r.x != o.x0) + (r.y != o.x1) + (r.z != o.x2) + (r.w != o.x3);
  }
  if (local) atomicAdd(bad, local);
}

}  // namespace

// words that differ over n draws (4 words each); -1 on a CUDA error
extern "C" long long philox_mismatches(unsigned long long n, unsigned long long seed) {
  unsigned long long *d = nullptr, h = 0;
  if (cudaMalloc(&d, sizeof(*d)) != cudaSuccess) return -1;
  cudaMemset(d, 0, sizeof(*d));
  philox_check_kernel<<<608, 256>>>(n, seed, d);
  cudaError_t e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? (long long)h : -1;
}
