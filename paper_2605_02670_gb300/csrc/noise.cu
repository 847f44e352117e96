// Lumped-mass white noise b = M_L^{1/2} xi (Eq. wh_def with the diagonal
// factor of Sec. 2.5): O(N), one Philox4x32-10 block per four DOFs.
//
// Philox4x32-10 follows its published definition (Salmon et al., SC'11):
// ten rounds of two 32x32->64 multiplies with M0 = 0xD2511F53 and
// M1 = 0xCD9E8D57, the key bumped by (0x9E3779B9, 0xBB67AE85) between rounds.
// Key = (seed lo32, seed hi32); counter = (q lo32, q hi32, s, 0) for DOFs
// 4q..4q+3 of sample s. Uniform u = (word + 1/2) 2^-32; Box-Muller on word
// pairs (0,1) and (2,3).
//
// HBM-bound: each thread writes four values and reads four mass factors.
#include "grf_internal.h"

namespace grf {
namespace {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // high and low words of the 32 x 32 -> 64-bit products as two 32-bit
    // multiplies each (a 64-bit product is issued to the FP64 pipe, which is
    // narrow on GB300)
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 noise_block(uint64_t seed, uint64_t q, uint32_t s) {
  return philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), s, 0u), (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

__device__ __forceinline__ void box_muller(uint32_t xa, uint32_t xb, double& n0, double& n1) {
  const double ua = ((double)xa + 0.5) * 0x1p-32;
  const double ub = ((double)xb + 0.5) * 0x1p-32;
  const double r = sqrt(-2.0 * log(ua));
  double sn, cs;
  sincospi(2.0 * ub, &sn, &cs);
  n0 = r * cs;
  n1 = r * sn;
}

// FP32 Box-Muller of the mixed-precision path: the hardware base-2
// logarithm, square root and sine/cosine (one special-function instruction
// each; their errors leave the normals within ~1e-6 relative in the L2 sense,
// far inside the FP32 sweeps' tolerance; the uint32 words stay bit-exact).
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void box_muller(uint32_t xa, uint32_t xb, float& n0, float& n1) {
  const float ua = fmaf((float)xa, 0x1p-32f, 0x1p-33f);
  const float ub = fmaf((float)xb, 0x1p-32f, 0x1p-33f);
  // -2 ln u = (-2 ln 2) log2 u >= 0 (u <= 1 after rounding)
  const float r = sqrt_approx(-1.3862943611198906f * __log2f(ua));
  float sn, cs;
  __sincosf(6.2831853071795865f * ub, &sn, &cs);
  n0 = r * cs;
  n1 = r * sn;
}

// Each thread keeps one sample s and walks the Philox blocks q of its row
// group: a CTA covers SB = min(S, 1024) samples (blockIdx.y picks the sample
// chunk) and blockDim / SB rows, so a warp writes whole rows b[j][s0..s0+31]
// and no thread divides per block.
// sml_f: the FP32 mass factors for T = float (one FP64 -> FP32 conversion per
// element would run on GB300's narrow FP64 pipe and bound the kernel).
template <typename T>
__global__ void noise_minor_kernel(DevGraph g, uint64_t seed, const uint64_t* seed_dev, int64_t S,
                                   int32_t SB, T* __restrict__ b,
                                   const float* __restrict__ sml_f) {
  if (seed_dev) seed = *seed_dev;
  const int64_t nq = (g.n + 3) / 4;
  const int32_t rows = blockDim.x / SB;  // Philox blocks per CTA pass
  const int32_t qi = threadIdx.x / SB;
  const int64_t s = (int64_t)blockIdx.y * SB + threadIdx.x % SB;
  if (qi >= rows || s >= S) return;
  const int64_t nfull = g.n / 4;  // blocks of four DOFs inside the vector
  const int64_t step = (int64_t)gridDim.x * rows;
  for (int64_t q = (int64_t)blockIdx.x * rows + qi; q < nq; q += step) {
    const uint4 w = noise_block(seed, (uint64_t)q, (uint32_t)s);
    T n[4];
    box_muller(w.x, w.y, n[0], n[1]);
    box_muller(w.z, w.w, n[2], n[3]);
    T* p = b + 4 * q * S + s;
    if (sizeof(T) == 4 && sml_f && q < nfull) {
      // the block's four mass factors in one 16-byte load (4 q is a multiple of 4)
      const float4 f = __ldg(reinterpret_cast<const float4*>(sml_f) + q);
      p[0] = (T)(f.x * (float)n[0]);
      p[S] = (T)(f.y * (float)n[1]);
      p[2 * S] = (T)(f.z * (float)n[2]);
      p[3 * S] = (T)(f.w * (float)n[3]);
      continue;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = 4 * q + k;
      if (j < g.n) {
        if (sizeof(T) == 4 && sml_f)
          p[k * S] = (T)(sml_f[j] * (float)n[k]);
        else
          p[k * S] = (T)g.sqrt_ml[j] * n[k];
      }
    }
  }
}

__global__ void noise_major_kernel(DevGraph g, uint64_t seed, int64_t S, void* out, int raw) {
  const int64_t nq = (g.n + 3) / 4;
  const int64_t total = nq * S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / nq;
    const int64_t q = t - s * nq;
    const uint4 w = noise_block(seed, (uint64_t)q, (uint32_t)s);
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
    double n[4];
    if (!raw) {
      box_muller(w.x, w.y, n[0], n[1]);
      box_muller(w.z, w.w, n[2], n[3]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = 4 * q + k;
      if (j >= g.n) break;
      if (raw)
        static_cast<uint32_t*>(out)[s * g.n + j] = words[k];
      else
        static_cast<double*>(out)[s * g.n + j] = g.sqrt_ml[j] * n[k];
    }
  }
}

int grid_for(int64_t total, int threads) {
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > sm_count() * 64) blocks = sm_count() * 64;
  return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace

template <typename T>
void launch_noise_minor(const DevGraph& g, uint64_t seed, int64_t S, T* b, cudaStream_t st,
                        const uint64_t* seed_dev, const float* sqrt_ml_f) {
  // SB samples per CTA, blockDim a multiple of SB (at least 256 threads when S allows)
  const int32_t SB = (int32_t)(S < 1024 ? S : 1024);
  const int32_t rows = SB >= 256 ? 1 : (256 + SB - 1) / SB;
  const int threads = rows * SB;
  const int64_t nq = (g.n + 3) / 4;
  int64_t bx = (nq + rows - 1) / rows;
  const int64_t by = (S + SB - 1) / SB;
  int64_t cap = sm_count() * 32 / by;
  if (cap < 1) cap = 1;
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  noise_minor_kernel<T><<<dim3((unsigned)bx, (unsigned)by), threads, 0, st>>>(
      g, seed, seed_dev, S, SB, b, sqrt_ml_f);
}
template void launch_noise_minor<float>(const DevGraph&, uint64_t, int64_t, float*, cudaStream_t,
                                        const uint64_t*, const float*);
template void launch_noise_minor<double>(const DevGraph&, uint64_t, int64_t, double*,
                                         cudaStream_t, const uint64_t*, const float*);

void launch_noise_major(const DevGraph& g, uint64_t seed, int64_t S, void* out, bool raw,
                        cudaStream_t st) {
  const int64_t total = ((g.n + 3) / 4) * S;
  noise_major_kernel<<<grid_for(total, 256), 256, 0, st>>>(g, seed, S, out, raw ? 1 : 0);
}

}  // namespace grf
