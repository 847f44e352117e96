// Spectral edge interiors on the tensor cores (mixed precision; Sec. 3, Phase 3,
// Eq. local_reduced_schur through the sine basis of spectral.cu).
//
// For one edge (m interior nodes) and 16 samples both dense contractions of the
// condensation are matrix products:
//   forward transform  bh = Phi b,              Phi_ji = sin(pi j i / (m+1)) sqrt(2/(m+1)),
//   end values         e1_l = sum_j bt_j / mu_jl,   em_l = sum_j (-1)^(j+1) bt_j / mu_jl,
//                      bt_j = phi_j bh_j,  mu_jl = delta_l + 4 sin^2(pi j / (2(m+1))).
// Both run as warp-level mma.sync m16n8k8 with TF32 operands in three terms
// (a_hi b_hi + a_hi b_lo + a_lo b_hi, x_hi = tf32(x), x_lo = tf32(x - x_hi)),
// which keeps the products to about 2^-21 relative: FP32 accuracy for the
// 1e-4 field tolerance. The left operand is generated in registers: the sines
// by rotation along the contraction index (re-anchored from a table every 16
// steps), 1 / mu_jl by one SFU reciprocal per element. The right operand
// (noise rows, bt) is staged in shared memory.
//
// Fragment layout of m16n8k8 (TF32): with g = lane / 4, t = lane % 4, A (16x8,
// row major) holds a0 = A[g][t], a1 = A[g+8][t], a2 = A[g][t+4], a3 = A[g+8][t+4];
// B (8x8, column major) b0 = B[t][g], b1 = B[t+4][g]; C (16x8) c0 = C[g][2t],
// c1 = C[g][2t+1], c2 = C[g+8][2t], c3 = C[g+8][2t+1].
#include <cuda_runtime.h>

#include "grf_internal.h"

namespace grf {
namespace {

constexpr int kSG = 16;  // samples per unit

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x = hi + lo with hi rounded to TF32; lo goes in as FP32 bits and the tensor
// core uses its leading TF32 bits (error below 2^-21 |x|)
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d[0] += A_hi B_hi, d[1] += A_hi B_lo, d[2] += A_lo B_hi (B already split):
// three independent accumulators, summed by the caller, so that consecutive
// tensor instructions do not wait on each other
__device__ __forceinline__ void mma3(float (&d)[3][4], const uint32_t (&ah)[4],
                                     const uint32_t (&al)[4], uint32_t bh0, uint32_t bh1,
                                     uint32_t bl0, uint32_t bl1) {
  mma_tf32(d[0], ah, bh0, bh1);
  mma_tf32(d[1], ah, bl0, bl1);
  mma_tf32(d[2], al, bh0, bh1);
}

// sin / cos (pi k / (m+1)) for k < 2(m+1); sig_j = 4 sin^2(pi (j+1) / (2(m+1))),
// j < mpad (finite beyond m: those modes meet zero rows).
__device__ __forceinline__ void tables(int32_t m, int32_t mpad, float* tab, float* ctab,
                                       float* sig) {
  const int32_t P = 2 * (m + 1);
  for (int32_t k = threadIdx.x; k < P; k += blockDim.x) {
    float sn, cs;
    sincospif((float)k / (float)(m + 1), &sn, &cs);
    tab[k] = sn;
    ctab[k] = cs;
  }
  for (int32_t j = threadIdx.x; j < mpad; j += blockDim.x) {
    const float sh = 2.f * sinpif((float)(j + 1) / (float)(2 * (m + 1)));
    sig[j] = sh * sh;
  }
}

// Y[16 x 16] tile of Phi X for modes 16 mt .. 16 mt + 15 (unscaled), X rows in
// shared memory [mpad][16] split into TF32 hi and lo parts (rows >= m zero).
// acc[nt][..] holds samples 8 nt ..
__device__ __forceinline__ void dst_tile(int32_t m, int32_t mpad, int mt, int lane,
                                         const float* tab, const float* ctab, const uint32_t* Xh,
                                         const uint32_t* Xl, float (&acc)[2][4]) {
  const int g = lane >> 2, t = lane & 3;
  const int32_t P = 2 * (m + 1);
  const int32_t j1 = 16 * mt + g + 1, j2 = j1 + 8;  // 1-based modes of this thread's rows
  // rotation per 8 columns: angle 8 pi j / (m+1)
  const int32_t r1 = (8 * j1) % P, r2 = (8 * j2) % P;
  const float c81 = ctab[r1], s81 = tab[r1], c82 = ctab[r2], s82 = tab[r2];
  float cs[4], sn[4];  // states of a0..a3: (j1, i1), (j2, i1), (j1, i2), (j2, i2)
  float d[2][3][4];
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k) d[nt][q][k] = 0.f;
  const int32_t nkt = mpad / 8;
  for (int32_t kt = 0; kt < nkt; ++kt) {
    if ((kt & 15) == 0) {  // re-anchor from the tables
      const int32_t i1 = 8 * kt + t + 1, i2 = i1 + 4;
      const int32_t k0 = (int32_t)(((int64_t)j1 * i1) % P), k1 = (int32_t)(((int64_t)j2 * i1) % P);
      const int32_t k2 = (int32_t)(((int64_t)j1 * i2) % P), k3 = (int32_t)(((int64_t)j2 * i2) % P);
      cs[0] = ctab[k0]; sn[0] = tab[k0];
      cs[1] = ctab[k1]; sn[1] = tab[k1];
      cs[2] = ctab[k2]; sn[2] = tab[k2];
      cs[3] = ctab[k3]; sn[3] = tab[k3];
    }
    uint32_t ah[4], al[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) split_tf32(sn[k], ah[k], al[k]);
    const size_t r0 = (size_t)(8 * kt + t) * kSG + g, r1 = r0 + 4 * kSG;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
      mma3(d[nt], ah, al, Xh[r0 + 8 * nt], Xh[r1 + 8 * nt], Xl[r0 + 8 * nt], Xl[r1 + 8 * nt]);
    // advance the columns by 8
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float c8 = (k & 1) ? c82 : c81, s8 = (k & 1) ? s82 : s81;
      const float c = fmaf(cs[k], c8, -sn[k] * s8);
      sn[k] = fmaf(sn[k], c8, cs[k] * s8);
      cs[k] = c;
    }
  }
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[nt][k] = d[nt][0][k] + (d[nt][1][k] + d[nt][2][k]);
}

template <int NW>
__host__ __device__ constexpr size_t cond_mma_floats(int32_t mmax, int32_t L) {
  const size_t mp = ((size_t)mmax + 7) / 8 * 8;
  return 2 * (mp + 8) * kSG + 4 * ((size_t)mmax + 1) + (mp + 8) + (size_t)L + 8;
}

// Forward transform of the edge's noise (written to bhat) and the two end
// values of T_l^-1 b_I for every node, added into gvec. One CTA per (edge,
// 16 samples); warps split the 16-row tiles.
template <int NW>
__global__ void __launch_bounds__(32 * NW)
    spec_condense_mma_kernel(DevGraph g, DevNodes nd, int64_t S, const float* __restrict__ b,
                             const int32_t* __restrict__ edges, int32_t n_edges, int32_t mmax,
                             float* __restrict__ bhat, double* __restrict__ gvec) {
  extern __shared__ __align__(16) float sm[];
  const int32_t mpmax = (mmax + 7) / 8 * 8;
  // [mpad][16] TF32 hi and lo parts: the noise rows, after the transform phi_j bh_j
  uint32_t* bsh = reinterpret_cast<uint32_t*>(sm);
  uint32_t* bsl = bsh + ((size_t)mpmax + 8) * kSG;
  float* tab = reinterpret_cast<float*>(bsl + ((size_t)mpmax + 8) * kSG);  // [2 (mmax + 1)]
  float* ctab = tab + 2 * ((size_t)mmax + 1);  // [2 (mmax + 1)]
  float* sig = ctab + 2 * ((size_t)mmax + 1);  // [mpad + 8]
  float* dls = sig + mpmax + 8;                // [L]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gq = lane >> 2, tq = lane & 3;
  const int64_t nsg = (S + kSG - 1) / kSG;
  const int64_t units = (int64_t)n_edges * nsg;
  const int32_t L = nd.L;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int32_t e = edges[u / nsg];
    const int64_t s0 = (u % nsg) * kSG;
    const int32_t m = g.nel[e] - 1;  // 1 <= m <= mmax for binned edges
    const int32_t mpad = (m + 7) / 8 * 8;
    const int64_t off = g.ioff[e];
    const int kv = (int)(S - s0 < kSG ? S - s0 : kSG);
    const double h = g.he[e];
    const float h2f = (float)(h * h);
    __syncthreads();  // the previous unit is done with the shared arrays
    tables(m, mpad + 8, tab, ctab, sig);
    for (int32_t l = threadIdx.x; l < L; l += blockDim.x) dls[l] = nd.shift[l] * h2f;
    const float* src = b + (g.nv + off) * S + s0;
    for (int32_t k = threadIdx.x; k < mpad * kSG; k += blockDim.x) {
      const int32_t i = k / kSG, c = k - i * kSG;
      const float x = (i < m && c < kv) ? src[(int64_t)i * S + c] : 0.f;
      split_tf32(x, bsh[k], bsl[k]);
    }
    __syncthreads();
    const float scale = sqrtf(2.f / (float)(m + 1));
    // forward transform, 16 modes per warp tile
    const int nmt = (m + 15) / 16;
    for (int mt = warp; mt < nmt; mt += NW) {
      float acc[2][4];
      dst_tile(m, mpad, mt, lane, tab, ctab, bsh, bsl, acc);
#pragma unroll
      for (int hrow = 0; hrow < 2; ++hrow) {
        const int32_t j = 16 * mt + gq + 8 * hrow;  // 0-based mode
        if (j < m) {
          float* bo = bhat + (off + j) * S + s0;
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            const int s = 8 * nt + 2 * tq;
            if (s < kv) bo[s] = scale * acc[nt][2 * hrow];
            if (s + 1 < kv) bo[s + 1] = scale * acc[nt][2 * hrow + 1];
          }
        }
      }
    }
    __syncthreads();  // every transform tile is in bhat; the noise rows are done
    // phi_j bh_j, split, over the noise rows, modes by parity: rows [0, mh) hold
    // the even 0-based modes 2r, rows [mh, 2 mh) the odd ones 2r + 1 (modes >= m
    // and samples >= kv zero)
    const int32_t mh = ((m + 1) / 2 + 7) / 8 * 8;
    for (int32_t k = threadIdx.x; k < 2 * mh * kSG; k += blockDim.x) {
      const int32_t row = k / kSG, c = k - row * kSG;
      const int32_t j = row < mh ? 2 * row : 2 * (row - mh) + 1;
      const float x = (j < m && c < kv)
                          ? scale * tab[(j + 1) % (2 * (m + 1))] * bhat[(off + j) * S + s0 + c]
                          : 0.f;
      split_tf32(x, bsh[k], bsl[k]);
    }
    __syncthreads();
    // end values (T^-1 b_I)_1 = O + E next to edge_u and (T^-1 b_I)_m = O - E
    // next to edge_v, O / E the sums over odd / even 1-based modes j of
    // phi_j bh_j / mu_jl: rows = nodes l (16 per tile), columns = 16 samples
    const int nlt = (L + 15) / 16;
    const int32_t va = g.eu[e], vb = g.ev[e];
    for (int lt = warp; lt < nlt; lt += NW) {
      const int32_t l1 = 16 * lt + gq, l2 = l1 + 8;
      const bool on1 = l1 < L, on2 = l2 < L;
      const float d1 = on1 ? dls[l1] : 1.f, d2 = on2 ? dls[l2] : 1.f;
      float acc[2][2][4];  // [parity][nt]
      float d[2][2][3][4];
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) d[p][nt][q][k] = 0.f;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        for (int32_t kt = 0; kt < mh / 8; ++kt) {
          const int32_t ra = 8 * kt + tq, rb = ra + 4;  // rows of this parity
          const float sa = sig[2 * ra + p], sb = sig[2 * rb + p];
          float av[4];
          av[0] = on1 ? __fdividef(1.f, d1 + sa) : 0.f;
          av[1] = on2 ? __fdividef(1.f, d2 + sa) : 0.f;
          av[2] = on1 ? __fdividef(1.f, d1 + sb) : 0.f;
          av[3] = on2 ? __fdividef(1.f, d2 + sb) : 0.f;
          uint32_t ah[4], al[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) split_tf32(av[k], ah[k], al[k]);
          const size_t r0 = (size_t)(p * mh + ra) * kSG + gq, r1 = r0 + 4 * kSG;
#pragma unroll
          for (int nt = 0; nt < 2; ++nt)
            mma3(d[p][nt], ah, al, bsh[r0 + 8 * nt], bsh[r1 + 8 * nt], bsl[r0 + 8 * nt],
                 bsl[r1 + 8 * nt]);
        }
      }
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int k = 0; k < 4; ++k)
            acc[p][nt][k] = d[p][nt][0][k] + (d[p][nt][1][k] + d[p][nt][2][k]);
#pragma unroll
      for (int hrow = 0; hrow < 2; ++hrow) {
        const int32_t l = hrow ? l2 : l1;
        if (l >= L) continue;
        double* gl = gvec + ((int64_t)l * S + s0) * g.nv;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int s = 8 * nt + 2 * tq + k;
            if (s < kv) {
              const float o = acc[0][nt][2 * hrow + k], ev = acc[1][nt][2 * hrow + k];
              atomicAdd(gl + (int64_t)s * g.nv + va, (double)(o + ev));
              atomicAdd(gl + (int64_t)s * g.nv + vb, (double)(o - ev));
            }
          }
        }
      }
    }
  }
}

int grid_units(int64_t units) {
  int64_t b = units < sm_count() * 16 ? units : sm_count() * 16;
  return b < 1 ? 1 : (int)b;
}

template <int NW>
void condense_mma_bin(const DevGraph& g, const DevNodes& nd, int64_t S, const float* b,
                      const int32_t* e, int32_t n, int32_t mmax, float* bhat, double* gvec,
                      cudaStream_t st) {
  const size_t smem = cond_mma_floats<NW>(mmax, nd.L) * sizeof(float);
  cudaFuncSetAttribute(spec_condense_mma_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  const int64_t units = (int64_t)n * ((S + kSG - 1) / kSG);
  spec_condense_mma_kernel<NW><<<grid_units(units), 32 * NW, smem, st>>>(g, nd, S, b, e, n, mmax,
                                                                       bhat, gvec);
}

}  // namespace

int launch_spec_condense_mma(const DevGraph& g, const DevNodes& nd, int64_t S, const float* b,
                             const int32_t* bin_edges, const int32_t* bin_count, float* bhat,
                             double* gvec, cudaStream_t st) {
  int32_t mmax[16];
  const int nb = spec_bins(mmax);
  const int32_t* e = bin_edges;
  int launches = 0;
  for (int i = 0; i < nb; ++i) {
    const int32_t n = bin_count[i];
    if (n > 0) {
      if (mmax[i] <= 256)
        condense_mma_bin<4>(g, nd, S, b, e, n, mmax[i], bhat, gvec, st);
      else
        condense_mma_bin<8>(g, nd, S, b, e, n, mmax[i], bhat, gvec, st);
      ++launches;
    }
    e += n;
  }
  return launches;
}

}  // namespace grf
