// Test helper (not part of the library): Philox4x32-10 blocks drawn through
// cuRAND's device API, to cross-check the sampler's own counter-based
// generator against an independent implementation of the same published
// definition. curand_init(seed, subsequence = s, offset = 4 q) starts the
// stream at key (seed lo32, seed hi32) and counter (q lo32, q hi32, s lo32,
// s hi32); the first curand4() call returns that block's four words.
// Compiled by tests/test_gpu_parity.py into a temporary directory.
#include <cstdint>

#include <curand_kernel.h>

namespace {

__global__ void curand_blocks_kernel(unsigned long long seed, const int32_t* sample,
                                     const int64_t* block, int64_t n, int32_t* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed, (unsigned long long)(uint32_t)sample[i], 4ull * (unsigned long long)block[i],
              &st);
  const uint4 r = curand4(&st);
  out[4 * i + 0] = (int32_t)r.x;
  out[4 * i + 1] = (int32_t)r.y;
  out[4 * i + 2] = (int32_t)r.z;
  out[4 * i + 3] = (int32_t)r.w;
}

}  // namespace

// sample: device int32 [n] (sample index s >= 0); block: device int64 [n]
// (block index q >= 0); out: device int32 [n][4]. Returns the CUDA error code of
// the launch and the synchronisation (0 on success).
extern "C" int curand_philox_blocks(unsigned long long seed, const int32_t* sample,
                                    const int64_t* block, int64_t n, int32_t* out) {
  if (n <= 0) return 0;
  const int threads = 128;
  const int64_t blocks = (n + threads - 1) / threads;
  curand_blocks_kernel<<<(unsigned)blocks, threads>>>(seed, sample, block, n, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  return (int)cudaDeviceSynchronize();
}
