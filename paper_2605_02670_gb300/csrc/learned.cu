// Learned BB^T preconditioner for the vertex Schur systems (Phase 4): a
// message-passing network over the vertex graph maps per-vertex features of
// the Jacobi-scaled system S_hat = D^-1/2 S D^-1/2 to a sparse factor
//   B = diag(exp(s)) + N  (N on the incidence pattern),
// and PCG uses z = B B^T r. The network (3 message-passing layers, width 64)
// runs its dense layers on the tensor cores: BF16 operands, FP32
// accumulation (mma.sync m16n8k16), for inference, input gradients and weight
// gradients; aggregation, heads, loss and the optimiser run on CUDA cores.
//
//   x_v = [1, log(1+deg)/3, sig, amax, sig^2, tanh(log t / 20), sig/deg, 0]
//         (a_k = -S_hat_vw per incidence k of v, sig = sum a_k, amax = max a_k)
//   h0 = relu(x W0 + b0);  h_i = relu([h_{i-1}, m_i] W_i + b_i),
//   m_i(v) = sum_k a_k h_{i-1}(nbr k);  s_v = h3 . ws + cs;
//   n_k = a_k (h3_v . u + h3_w . up + cn)  (k: v -> w).
// Loss over pairs (r, e), S_hat e = r: mean (B B^T r - e)^T S_hat (B B^T r - e)
// / (r^T e). With zero heads B = I: plain Jacobi, which is the fallback.
#include <cuda_bf16.h>

#include "grf_internal.h"

namespace grf {
namespace lp {

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D = A (16x16, row) x B (16x8, col) + D, BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[M x N] = A[M x K] B[K x N] (+ bias, relu). A: BF16 row-major (lda), B: BF16
// row-major [K x N]; K % 16 == 0, N % 8 == 0, N <= 128, K <= 128. Outputs: FP32 C
// (ldc, may be null) and/or a BF16 copy D (ldd, may be null). One warp per 16
// rows; B staged in shared memory.
template <int N>
__global__ void __launch_bounds__(128) gemm_kernel(int64_t M, int K,
                                                   const __nv_bfloat16* __restrict__ A, int lda,
                                                   const __nv_bfloat16* __restrict__ B,
                                                   const float* __restrict__ bias, int relu,
                                                   float* __restrict__ C, int ldc,
                                                   __nv_bfloat16* __restrict__ D, int ldd) {
  __shared__ __nv_bfloat16 sb[128 * N];
  for (int i = threadIdx.x; i < K * N; i += blockDim.x) sb[i] = B[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, tq = lane & 3;
  for (int64_t r0 = ((int64_t)blockIdx.x * 4 + warp) * 16; r0 < M;
       r0 += (int64_t)gridDim.x * 64) {
    float acc[N / 8][4];
#pragma unroll
    for (int nt = 0; nt < N / 8; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
    const int64_t ra = r0 + gq, rb = r0 + gq + 8;
    for (int kk = 0; kk < K; kk += 16) {
      uint32_t a[4];
      const __nv_bfloat16 z = __float2bfloat16(0.f);
      auto ld = [&](int64_t r, int c) -> uint32_t {
        if (r >= M) return pack_raw(z, z);
        const __nv_bfloat16* p = A + r * lda + c;
        return pack_raw(p[0], p[1]);
      };
      a[0] = ld(ra, kk + 2 * tq);
      a[1] = ld(rb, kk + 2 * tq);
      a[2] = ld(ra, kk + 2 * tq + 8);
      a[3] = ld(rb, kk + 2 * tq + 8);
#pragma unroll
      for (int nt = 0; nt < N / 8; ++nt) {
        const int n = nt * 8 + gq;
        uint32_t b[2];
        b[0] = pack_raw(sb[(kk + 2 * tq) * N + n], sb[(kk + 2 * tq + 1) * N + n]);
        b[1] = pack_raw(sb[(kk + 2 * tq + 8) * N + n], sb[(kk + 2 * tq + 9) * N + n]);
        mma16816(acc[nt], a, b);
      }
    }
#pragma unroll
    for (int nt = 0; nt < N / 8; ++nt) {
      const int c0 = nt * 8 + 2 * tq;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t r = h ? rb : ra;
        if (r >= M) continue;
        float v0 = acc[nt][2 * h], v1 = acc[nt][2 * h + 1];
        if (bias) {
          v0 += bias[c0];
          v1 += bias[c0 + 1];
        }
        if (relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (C) {
          C[r * ldc + c0] = v0;
          C[r * ldc + c0 + 1] = v1;
        }
        if (D) {
          D[r * ldd + c0] = __float2bfloat16(v0);
          D[r * ldd + c0 + 1] = __float2bfloat16(v1);
        }
      }
    }
  }
}

// G[K x 64] += A^T[K x M] Y[M x 64]: weight gradients. A: BF16 [M x K] (lda),
// Y: BF16 [M x 64] (ldy). One warp per 16-row tile of K; the CTA walks a chunk
// of M rows and adds its partial product atomically.
// Only rows k < kout of G are written.
__global__ void __launch_bounds__(256) gemm_tn_kernel(int64_t M, int K,
                                                      const __nv_bfloat16* __restrict__ A,
                                                      int lda,
                                                      const __nv_bfloat16* __restrict__ Y,
                                                      int ldy, float* __restrict__ G,
                                                      int64_t chunk, int kout) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, tq = lane & 3;
  const int k0 = warp * 16;
  if (k0 >= K) return;
  const int64_t m_begin = (int64_t)blockIdx.x * chunk;
  const int64_t m_end = m_begin + chunk < M ? m_begin + chunk : M;
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
  const __nv_bfloat16 z = __float2bfloat16(0.f);
  for (int64_t mm = m_begin; mm < m_end; mm += 16) {
    // A operand = A^T: element (row k, col m) = A[m][k]
    auto at = [&](int k, int64_t m) -> __nv_bfloat16 { return m < m_end ? A[m * lda + k] : z; };
    uint32_t a[4];
    a[0] = pack_raw(at(k0 + gq, mm + 2 * tq), at(k0 + gq, mm + 2 * tq + 1));
    a[1] = pack_raw(at(k0 + gq + 8, mm + 2 * tq), at(k0 + gq + 8, mm + 2 * tq + 1));
    a[2] = pack_raw(at(k0 + gq, mm + 2 * tq + 8), at(k0 + gq, mm + 2 * tq + 9));
    a[3] = pack_raw(at(k0 + gq + 8, mm + 2 * tq + 8), at(k0 + gq + 8, mm + 2 * tq + 9));
    auto yv = [&](int64_t m, int n) -> __nv_bfloat16 { return m < m_end ? Y[m * ldy + n] : z; };
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int n = nt * 8 + gq;
      uint32_t b[2];
      b[0] = pack_raw(yv(mm + 2 * tq, n), yv(mm + 2 * tq + 1, n));
      b[1] = pack_raw(yv(mm + 2 * tq + 8, n), yv(mm + 2 * tq + 9, n));
      mma16816(acc[nt], a, b);
    }
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int c0 = nt * 8 + 2 * tq;
    if (k0 + gq < kout) {
      atomicAdd(&G[(k0 + gq) * 64 + c0], acc[nt][0]);
      atomicAdd(&G[(k0 + gq) * 64 + c0 + 1], acc[nt][1]);
    }
    if (k0 + gq + 8 < kout) {
      atomicAdd(&G[(k0 + gq + 8) * 64 + c0], acc[nt][2]);
      atomicAdd(&G[(k0 + gq + 8) * 64 + c0 + 1], acc[nt][3]);
    }
  }
}

__device__ __forceinline__ float coupling(const float* offv_t, int64_t k) { return -offv_t[k]; }

// Features of node j (global node l = lnode[j]) into X0[j*V + v][0..15] (BF16).
__global__ void features_kernel(DevGraph g, int32_t Lb, const int32_t* __restrict__ lnode,
                                const float* __restrict__ offv_t, const double* __restrict__ alpha,
                                const double* __restrict__ gamma, __nv_bfloat16* __restrict__ X0) {
  const int64_t total = (int64_t)Lb * g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / g.nv;
    const int32_t v = (int32_t)(t - j * g.nv);
    const int64_t l = lnode[j];
    float sig = 0.f, amax = 0.f;
    for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
      const float a = coupling(offv_t, l * ne2 + k);
      sig += a;
      amax = fmaxf(amax, a);
    }
    const float deg = (float)(g.vptr[v + 1] - g.vptr[v]);
    const double al = alpha[l], ga = gamma[l];
    const float lt = al > 0 ? (float)log(ga / al) : 1e30f;
    float f[16] = {1.f, log1pf(deg) / 3.f, sig, amax, sig * sig, tanhf(lt / 20.f),
                   sig / fmaxf(deg, 1.f), 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 16; ++c) X0[t * 16 + c] = __float2bfloat16(f[c]);
  }
}

// m(j, v)[c] = sum over incidences k of v of a_k hin(j, nbr k)[c], 64 channels,
// one warp per (j, v). hin FP32 (ldi, column offset ci); result to BF16 (ldo,
// column offset co) or added to FP32 (add != 0).
__global__ void aggregate_kernel(DevGraph g, int32_t Lb, const int32_t* __restrict__ lnode,
                                 const float* __restrict__ offv_t, const float* __restrict__ hin,
                                 int ldi, int ci, const float* __restrict__ self, int lds,
                                 __nv_bfloat16* __restrict__ obf, float* __restrict__ of32,
                                 int ldo, int co) {
  const int64_t total = (int64_t)Lb * g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  const int lane = threadIdx.x & 31;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < total;
       t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t j = t / g.nv;
    const int32_t v = (int32_t)(t - j * g.nv);
    const int64_t l = lnode[j];
    float m0 = 0.f, m1 = 0.f;
    for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
      const float a = coupling(offv_t, l * ne2 + k);
      const float* row = hin + (j * g.nv + g.adj_nbr[k]) * ldi + ci;
      m0 += a * row[2 * lane];
      m1 += a * row[2 * lane + 1];
    }
    if (self) {  // FP32 result = self + aggregate
      m0 += self[t * lds + 2 * lane];
      m1 += self[t * lds + 2 * lane + 1];
    }
    if (obf) {
      obf[t * ldo + co + 2 * lane] = __float2bfloat16(m0);
      obf[t * ldo + co + 2 * lane + 1] = __float2bfloat16(m1);
    }
    if (of32) {
      of32[t * ldo + co + 2 * lane] = m0;
      of32[t * ldo + co + 2 * lane + 1] = m1;
    }
  }
}

// Heads: s, exp(s), alpha_v = h.u, beta_v = h.up for every (j, v); one warp each.
__global__ void heads_kernel(int64_t total, const float* __restrict__ h3,
                             const float* __restrict__ P, float* __restrict__ s,
                             float* __restrict__ es, float* __restrict__ al,
                             float* __restrict__ be) {
  const int lane = threadIdx.x & 31;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < total;
       t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const float h0 = h3[t * 64 + 2 * lane], h1 = h3[t * 64 + 2 * lane + 1];
    float a = h0 * P[kOffWs + 2 * lane] + h1 * P[kOffWs + 2 * lane + 1];
    float b = h0 * P[kOffU + 2 * lane] + h1 * P[kOffU + 2 * lane + 1];
    float c = h0 * P[kOffUp + 2 * lane] + h1 * P[kOffUp + 2 * lane + 1];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
      const float sv = a + P[kOffCs];
      s[t] = sv;
      es[t] = expf(sv);
      al[t] = b;
      be[t] = c;
    }
  }
}

// n(j, k) = a_k (alpha_v + beta_nbr + cn) for the incidences k of every v.
__global__ void offdiag_kernel(DevGraph g, int32_t Lb, const int32_t* __restrict__ lnode,
                               const float* __restrict__ offv_t, const float* __restrict__ al,
                               const float* __restrict__ be, const float* __restrict__ P,
                               float* __restrict__ n) {
  const int64_t total = (int64_t)Lb * g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / g.nv;
    const int32_t v = (int32_t)(t - j * g.nv);
    const int64_t l = lnode[j];
    for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k)
      n[j * ne2 + k] = coupling(offv_t, l * ne2 + k) *
                       (al[t] + be[j * g.nv + g.adj_nbr[k]] + P[kOffCn]);
  }
}

// One CTA per pair p (all pairs of node j, local node index pj[p]): loss and
// the gradients with respect to s and n (summed over pairs, atomics).
//   y = B^T r, z = B y, eps = z - e, q = S_hat eps, c = r.e,
//   L = eps.q / c / P,  gz = 2 q / c / P,  t = B^T gz,
//   ds_v += exp(s_v) (gz_v y_v + r_v t_v),  dn_k += gz_v y_w + r_v t_w.
__global__ void __launch_bounds__(256) loss_grad_kernel(
    DevGraph g, int64_t npairs, const int32_t* __restrict__ pj, const int64_t* __restrict__ slot,
    const int32_t* __restrict__ lnode, const float* __restrict__ offv_t,
    const float* __restrict__ R, const float* __restrict__ Ev,
    const float* __restrict__ es, const float* __restrict__ n, float* __restrict__ scratch,
    float* __restrict__ ds, float* __restrict__ dn, float* __restrict__ loss, float inv_p) {
  __shared__ double red[2][8];
  const int32_t nv = g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  for (int64_t p = blockIdx.x; p < npairs; p += gridDim.x) {
    const int64_t j = pj[p];
    const int64_t l = lnode[j];
    const int64_t sp = slot ? slot[p] : p;
    const float* r = R + sp * nv;
    const float* e = Ev + sp * nv;
    const float* esj = es + j * nv;
    const float* nj = n + j * ne2;
    const float* ov = offv_t + l * ne2;
    float* y = scratch + (size_t)blockIdx.x * 4 * nv;
    float* eps = y + nv;
    float* gz = eps + nv;
    float* tt = gz + nv;
    // y = B^T r: y_w = es_w r_w + sum over k' of w of n_{rev k'} r_{nbr k'}
    for (int32_t w = threadIdx.x; w < nv; w += blockDim.x) {
      float acc = esj[w] * r[w];
      for (int32_t k = g.vptr[w]; k < g.vptr[w + 1]; ++k)
        acc += nj[g.adj_rev[k]] * r[g.adj_nbr[k]];
      y[w] = acc;
    }
    __syncthreads();
    for (int32_t v = threadIdx.x; v < nv; v += blockDim.x) {
      float acc = esj[v] * y[v];
      for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) acc += nj[k] * y[g.adj_nbr[k]];
      eps[v] = acc - e[v];
    }
    __syncthreads();
    double part[2] = {0.0, 0.0};  // eps.q, r.e
    for (int32_t v = threadIdx.x; v < nv; v += blockDim.x) {
      float q = eps[v];
      for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) q += ov[k] * eps[g.adj_nbr[k]];
      gz[v] = q;
      part[0] += (double)eps[v] * q;
      part[1] += (double)r[v] * e[v];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      part[0] += __shfl_xor_sync(0xffffffffu, part[0], o);
      part[1] += __shfl_xor_sync(0xffffffffu, part[1], o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = part[0];
      red[1][threadIdx.x >> 5] = part[1];
    }
    __syncthreads();
    double eq = 0.0, c = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      eq += red[0][w];
      c += red[1][w];
    }
    // a pair whose r.e is not positive (S_hat is SPD, so only a corrupt pair)
    // contributes nothing; c is the same in every thread
    if (!(c > 0.0) || !isfinite(eq / c)) {
      __syncthreads();
      continue;
    }
    const float scale = (float)(2.0 / c) * inv_p;
    if (threadIdx.x == 0) atomicAdd(loss, (float)(eq / c) * inv_p);
    for (int32_t v = threadIdx.x; v < nv; v += blockDim.x) gz[v] *= scale;
    __syncthreads();
    for (int32_t w = threadIdx.x; w < nv; w += blockDim.x) {
      float acc = esj[w] * gz[w];
      for (int32_t k = g.vptr[w]; k < g.vptr[w + 1]; ++k)
        acc += nj[g.adj_rev[k]] * gz[g.adj_nbr[k]];
      tt[w] = acc;
    }
    __syncthreads();
    for (int32_t v = threadIdx.x; v < nv; v += blockDim.x) {
      atomicAdd(&ds[j * nv + v], esj[v] * (gz[v] * y[v] + r[v] * tt[v]));
      for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
        const int32_t w = g.adj_nbr[k];
        atomicAdd(&dn[j * ne2 + k], gz[v] * y[w] + r[v] * tt[w]);
      }
    }
    __syncthreads();
  }
}

// Heads backward: dalpha_v = sum_k a_k dn_k, dbeta_v = sum_k' a_k' dn_{rev k'},
// dh3 = ds ws + dalpha u + dbeta up, and the head weight gradients.
__global__ void heads_bwd_kernel(DevGraph g, int32_t Lb, const int32_t* __restrict__ lnode,
                                 const float* __restrict__ offv_t, const float* __restrict__ h3,
                                 const float* __restrict__ P, const float* __restrict__ ds,
                                 const float* __restrict__ dn, float* __restrict__ dh,
                                 float* __restrict__ G) {
  const int64_t total = (int64_t)Lb * g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  const int lane = threadIdx.x & 31;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < total;
       t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t j = t / g.nv;
    const int32_t v = (int32_t)(t - j * g.nv);
    const int64_t l = lnode[j];
    float dal = 0.f, dbe = 0.f;
    for (int32_t k = g.vptr[v] + lane; k < g.vptr[v + 1]; k += 32) {
      const float a = coupling(offv_t, l * ne2 + k);
      dal += a * dn[j * ne2 + k];
      dbe += a * dn[j * ne2 + g.adj_rev[k]];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dal += __shfl_xor_sync(0xffffffffu, dal, o);
      dbe += __shfl_xor_sync(0xffffffffu, dbe, o);
    }
    const float dsv = ds[t];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = 2 * lane + q;
      const float hv = h3[t * 64 + c];
      dh[t * 64 + c] = dsv * P[kOffWs + c] + dal * P[kOffU + c] + dbe * P[kOffUp + c];
      atomicAdd(&G[kOffWs + c], dsv * hv);
      atomicAdd(&G[kOffU + c], dal * hv);
      atomicAdd(&G[kOffUp + c], dbe * hv);
    }
    if (lane == 0) {
      atomicAdd(&G[kOffCs], dsv);
      atomicAdd(&G[kOffCn], dal);
    }
  }
}

// dA = dH * (H > 0) in BF16, and the bias gradient sum over rows.
__global__ void relu_bwd_kernel(int64_t M, const float* __restrict__ dH, const float* __restrict__ H,
                                __nv_bfloat16* __restrict__ dA, float* __restrict__ db) {
  __shared__ float part[64];
  if (threadIdx.x < 64) part[threadIdx.x] = 0.f;
  __syncthreads();
  const int64_t total = M * 64;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = H[i] > 0.f ? dH[i] : 0.f;
    dA[i] = __float2bfloat16(v);
    atomicAdd(&part[i & 63], v);
  }
  __syncthreads();
  if (threadIdx.x < 64) atomicAdd(&db[threadIdx.x], part[threadIdx.x]);
}

// FP32 master weights -> BF16 copies: W0 padded to 16 rows, W1..W3 and their
// transposes (for the input gradients).
__global__ void weights_bf16_kernel(const float* __restrict__ P, __nv_bfloat16* __restrict__ wb,
                                    __nv_bfloat16* __restrict__ wt) {
  const int total = 16 * 64 + 3 * 128 * 64;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    if (i < 16 * 64) {
      const int r = i / 64, c = i % 64;
      wb[i] = __float2bfloat16(r < kFeat ? P[kOffW0 + r * 64 + c] : 0.f);
    } else {
      const int li = (i - 16 * 64) / (128 * 64);
      const int o = (i - 16 * 64) % (128 * 64);
      const int r = o / 64, c = o % 64;
      const float w = P[layer_w_off(li + 1) + o];
      wb[i] = __float2bfloat16(w);
      wt[li * 128 * 64 + c * 128 + r] = __float2bfloat16(w);
    }
  }
}

__global__ void adam_kernel(int np, float* __restrict__ P, float* __restrict__ G,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    const float gi = G[i];
    m[i] = b1 * m[i] + (1.f - b1) * gi;
    v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
    P[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
    G[i] = 0.f;
  }
}

// Plain CG on S_hat x = g_hat (FP64, unit-diagonal scaled system, Jacobi-PCG on
// S) for system sys (node l = sys / S), recording (r_i, x_i) at every
// `stride`-th iteration (up to per_sys records, and only while
// ||r_i|| > 1e3 rtol ||g_hat||, so that x* - x_i is accurate to about 1e-3),
// until ||r|| <= rtol ||g_hat|| or max_iter. Afterwards the errors
// e_i = x* - x_i are formed. Both members of a pair are divided by ||r_i||
// (the loss does not depend on a common scale) and stored in FP32;
// count[sys] = records made.
__global__ void __launch_bounds__(256) record_pairs_kernel(
    DevGraph g, int64_t nsys, int64_t S, const double* __restrict__ diag,
    const double* __restrict__ offv, const double* __restrict__ gvec, double* __restrict__ work,
    double* __restrict__ xrec, float* __restrict__ Rout, float* __restrict__ Eout,
    double* __restrict__ rinv, int32_t* __restrict__ count, int per_sys, int stride,
    double rtol, int max_iter) {
  __shared__ double red[8];
  __shared__ double bc;
  const int32_t nv = g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  auto bsum = [&](double v) -> double {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
      bc = a;
    }
    __syncthreads();
    return bc;
  };
  for (int64_t sys = blockIdx.x; sys < nsys; sys += gridDim.x) {
    const int64_t l = sys / S;
    const double* D = diag + l * nv;
    const double* O = offv + l * ne2;
    double* x = work + (size_t)blockIdx.x * 4 * nv;
    double* r = x + nv;
    double* p = r + nv;
    double* q = p + nv;
    double gg = 0.0;
    for (int32_t v = threadIdx.x; v < nv; v += blockDim.x) {
      const double gh = gvec[sys * nv + v] / sqrt(D[v]);
      x[v] = 0.0;
      r[v] = gh;
      p[v] = gh;
      gg += gh * gh;
    }
    gg = bsum(gg);
    double rr = gg;
    int rec = 0;
    const double floor2 = 1e6 * rtol * rtol * gg;
    for (int it = 0; it <= max_iter; ++it) {
      if (it % stride == 0 && rec < per_sys && rr > floor2) {
        const double inv = rr > 0 ? 1.0 / sqrt(rr) : 0.0;
        float* Rr = Rout + ((size_t)sys * per_sys + rec) * nv;
        double* Xr = xrec + ((size_t)blockIdx.x * per_sys + rec) * nv;
        for (int32_t v = threadIdx.x; v < nv; v += blockDim.x) {
          Rr[v] = (float)(r[v] * inv);
          Xr[v] = x[v];
        }
        if (threadIdx.x == 0) rinv[(size_t)sys * per_sys + rec] = inv;
        ++rec;
      }
      if (!(rr > rtol * rtol * gg) || it == max_iter) break;
      __syncthreads();
      double pq = 0.0;
      for (int32_t v = threadIdx.x; v < nv; v += blockDim.x) {
        double y = p[v];
        const double sv = 1.0 / sqrt(D[v]);
        for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
          const int32_t w = g.adj_nbr[k];
          y += O[k] * sv / sqrt(D[w]) * p[w];
        }
        q[v] = y;
        pq += p[v] * y;
      }
      pq = bsum(pq);
      if (!(pq > 0.0)) break;
      const double al = rr / pq;
      double rn = 0.0;
      for (int32_t v = threadIdx.x; v < nv; v += blockDim.x) {
        x[v] += al * p[v];
        r[v] -= al * q[v];
        rn += r[v] * r[v];
      }
      rn = bsum(rn);
      const double be = rn / rr;
      rr = rn;
      for (int32_t v = threadIdx.x; v < nv; v += blockDim.x) p[v] = r[v] + be * p[v];
      __syncthreads();
    }
    __syncthreads();
    // e_i = (x* - x_i) / ||r_i||
    for (int i = 0; i < rec; ++i) {
      const double* Xr = xrec + ((size_t)blockIdx.x * per_sys + i) * nv;
      float* Er = Eout + ((size_t)sys * per_sys + i) * nv;
      const double sc = rinv[(size_t)sys * per_sys + i];
      for (int32_t v = threadIdx.x; v < nv; v += blockDim.x)
        Er[v] = (float)((x[v] - Xr[v]) * sc);
    }
    if (threadIdx.x == 0) count[sys] = rec;
    __syncthreads();
  }
}

int grid_for(int64_t total, int threads) {
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > sm_count() * 32) blocks = sm_count() * 32;
  return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace lp

using namespace lp;

void lp_weights_bf16(const float* P, __nv_bfloat16* wb, __nv_bfloat16* wt, cudaStream_t st) {
  weights_bf16_kernel<<<64, 256, 0, st>>>(P, wb, wt);
}

// Forward of Lb nodes. Buffers (rows M = Lb * V):
//   X0 [M x 16] BF16, H[0..3] [M x 64] FP32, Xc[0..2] [M x 128] BF16,
//   s, es, al, be [M] FP32, n [Lb x 2E] FP32.
int lp_forward(const DevGraph& g, int32_t Lb, const int32_t* lnode, const float* offv_t,
               const double* alpha, const double* gamma, const float* P,
               const __nv_bfloat16* wb, const LpActs& a, cudaStream_t st) {
  const int64_t M = (int64_t)Lb * g.nv;
  const int gb = (int)((M + 63) / 64 < sm_count() * 16 ? (M + 63) / 64 : sm_count() * 16);
  features_kernel<<<grid_for(M, 256), 256, 0, st>>>(g, Lb, lnode, offv_t, alpha, gamma, a.X0);
  // h0 = relu(x W0 + b0), also the left half of the layer-1 input
  gemm_kernel<64><<<gb, 128, 0, st>>>(M, 16, a.X0, 16, wb, P + kOffB0, 1, a.H[0], 64, a.Xc[0],
                                     128);
  for (int i = 1; i <= kLayers; ++i) {
    // right half: m_i = aggregate(h_{i-1})
    aggregate_kernel<<<grid_for(M * 32, 256), 256, 0, st>>>(g, Lb, lnode, offv_t, a.H[i - 1], 64,
                                                          0, nullptr, 0, a.Xc[i - 1], nullptr,
                                                          128, 64);
    __nv_bfloat16* next = i < kLayers ? a.Xc[i] : nullptr;
    gemm_kernel<64><<<gb, 128, 0, st>>>(M, 128, a.Xc[i - 1], 128, wb + 16 * 64 + (i - 1) * 8192,
                                       P + layer_w_off(i) + 8192, 1, a.H[i], 64, next, 128);
  }
  heads_kernel<<<grid_for(M * 32, 256), 256, 0, st>>>(M, a.H[kLayers], P, a.s, a.es, a.al, a.be);
  offdiag_kernel<<<grid_for(M, 256), 256, 0, st>>>(g, Lb, lnode, offv_t, a.al, a.be, P, a.n);
  return 4 + 2 * kLayers;
}

// Loss and gradient for npairs pairs of the Lb nodes just run forward; grads
// accumulate into G (FP32, kParams), loss into *loss.
void lp_backward(const DevGraph& g, int32_t Lb, const int32_t* lnode, const float* offv_t,
                 const float* P, const __nv_bfloat16* wt, const LpActs& a, int64_t npairs,
                 const int32_t* pj, const int64_t* slot, const float* R, const float* E,
                 float inv_p, const LpGrads& b, float* G, float* loss, cudaStream_t st) {
  const int64_t M = (int64_t)Lb * g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  cudaMemsetAsync(b.ds, 0, sizeof(float) * M, st);
  cudaMemsetAsync(b.dn, 0, sizeof(float) * Lb * ne2, st);
  int pblocks = (int)(npairs < b.max_pair_ctas ? npairs : b.max_pair_ctas);
  if (pblocks < 1) pblocks = 1;
  loss_grad_kernel<<<pblocks, 256, 0, st>>>(g, npairs, pj, slot, lnode, offv_t, R, E, a.es,
                                            a.n, b.scratch, b.ds, b.dn, loss, inv_p);
  heads_bwd_kernel<<<grid_for(M * 32, 256), 256, 0, st>>>(g, Lb, lnode, offv_t, a.H[kLayers], P,
                                                        b.ds, b.dn, b.dH, G);
  const int gb = (int)((M + 63) / 64 < sm_count() * 16 ? (M + 63) / 64 : sm_count() * 16);
  const int64_t chunk = 1024;
  const int cb = (int)((M + chunk - 1) / chunk);
  for (int i = kLayers; i >= 1; --i) {
    relu_bwd_kernel<<<grid_for(M * 64, 256), 256, 0, st>>>(M, b.dH, a.H[i], b.dA,
                                                         G + layer_w_off(i) + 8192);
    gemm_tn_kernel<<<cb, 256, 0, st>>>(M, 128, a.Xc[i - 1], 128, b.dA, 64,
                                       G + layer_w_off(i), chunk, 128);
    // dXc = dA W_i^T  [M x 128]
    gemm_kernel<128><<<gb, 128, 0, st>>>(M, 64, b.dA, 64, wt + (i - 1) * 8192, nullptr, 0, b.dX,
                                        128, nullptr, 0);
    // dh_{i-1} = dXc[:, :64] + aggregate(dXc[:, 64:])
    aggregate_kernel<<<grid_for(M * 32, 256), 256, 0, st>>>(g, Lb, lnode, offv_t, b.dX, 128, 64,
                                                          b.dX, 128, nullptr, b.dH, 64, 0);
  }
  relu_bwd_kernel<<<grid_for(M * 64, 256), 256, 0, st>>>(M, b.dH, a.H[0], b.dA, G + kOffB0);
  // dW0: the input has 16 columns, rows kFeat.. are padding and not written
  gemm_tn_kernel<<<cb, 256, 0, st>>>(M, 16, a.X0, 16, b.dA, 64, G + kOffW0, chunk, kFeat);
}

void lp_adam(float* P, float* G, float* m, float* v, float lr, int step, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<64, 256, 0, st>>>(kParams, P, G, m, v, lr, b1, b2, 1e-8f, c1, c2);
}

void lp_record_pairs(const DevGraph& g, int64_t nsys, int64_t S, const double* diag,
                     const double* offv, const double* gvec, double* work, double* xrec,
                     float* R, float* E, double* rinv, int32_t* count, int per_sys, int stride,
                     double rtol, int max_iter, int ctas, cudaStream_t st) {
  record_pairs_kernel<<<ctas, 256, 0, st>>>(g, nsys, S, diag, offv, gvec, work, xrec, R, E, rinv,
                                           count, per_sys, stride, rtol, max_iter);
}

}  // namespace grf
