// Edge-interior solves of the domain decomposition in the sine basis (mixed
// precision; Sec. 3, Phases 3 and 5, Eq. local_reduced_schur and Eq.
// internal_recovery evaluated through an exact change of basis).
//
// On edge e (m interior nodes, uniform mesh h_e) the interior block of
// A_l = alpha_l M_L + gamma_l K is c_l T_l with T_l = tridiag(-1, 2 + delta_l, -1).
// Every T_l is diagonalised by the same discrete sine transform (DST-I):
//   T_l = Phi diag(mu_jl) Phi,   Phi_ij = sqrt(2/(m+1)) sin(pi i j / (m+1)),
//   mu_jl = delta_l + 4 sin^2(pi j / (2(m+1))),   Phi Phi = I,
// and Phi e_1 = phi, Phi e_m = ((-1)^(j+1) phi_j), phi_j = Phi_1j. With
// bh = Phi b_I (one transform per edge and sample):
//   condensation:  (T_l^-1 b_I)_1 = O_l + E_l,  (T_l^-1 b_I)_m = O_l - E_l,
//                  O_l / E_l = sum over odd / even j of phi_j bh_j / mu_jl;
//   recovery:      U_I = sum_l T_l^-1 (sc_l b_I + xa_l e_1 + xb_l e_m) = Phi c,
//                  c_j = D_j bh_j + phi_j sum_l (xa_l + (-1)^(j+1) xb_l) / mu_jl,
//                  D_j = sum_l sc_l / mu_jl,
// where sc_l = w_l / c_l and xa_l = w_l u_a^(l), xb_l = w_l u_b^(l) are the
// weighted vertex values. The L tridiagonal solves per edge and sample of the
// Thomas form become a transform pair plus an (m x L) by (L x SG) contraction
// whose matrix 1 / mu_jl is generated on the fly; everything runs in FP32 with
// the node sums over at most L terms of one sign pattern per mode.
//
// One CTA per (edge, group of SG samples); the edge's rows, the sine table
// sin(pi k / (m+1)), k < 2(m+1), and the mode shifts 4 sin^2(pi j / (2(m+1)))
// live in shared memory. Edges are binned by m so that the shared-memory size
// of a launch fits its largest edge.
#include "grf_internal.h"

namespace grf {
namespace {

constexpr int kSpecLChunk = 128;  // nodes staged per pass in the recovery

// sin(pi k / (m+1)) and cos(pi k / (m+1)) for k < 2(m+1), the mode shifts
// sig_j = 4 sin^2(pi j / (2(m+1))), j = 1..m.
__device__ __forceinline__ void spec_tables(int32_t m, float* tab, float* ctab, float* sig) {
  const int32_t P = 2 * (m + 1);
  for (int32_t k = threadIdx.x; k < P; k += blockDim.x) {
    float sn, cs;
    sincospif((float)k / (float)(m + 1), &sn, &cs);
    tab[k] = sn;
    ctab[k] = cs;
  }
  for (int32_t j = threadIdx.x; j < m; j += blockDim.x) {
    const float sh = 2.f * sinpif((float)(j + 1) / (float)(2 * (m + 1)));
    sig[j] = sh * sh;
  }
}

// acc[q][s] = sum_{i=1..m} sin(pi i j_q / (m+1)) src[i-1][s] for the thread's QJ
// indices j_q (1-based; j_q = 0 gives zeros). The pair (cos, sin)(pi i j_q / (m+1))
// advances by a rotation through pi j_q / (m+1) and is re-read from the tables
// every 32 steps, so the rounding drift stays within a few dozen ulp; the rows
// of src are loaded once for the QJ indices.
template <int SG, int QJ>
__device__ __forceinline__ void dst_rows(int32_t m, const int32_t (&j)[QJ], const float* tab,
                                         const float* ctab, const float* src,
                                         float (&acc)[QJ][SG]) {
  const int32_t P = 2 * (m + 1);
  float c1[QJ], s1[QJ], cs[QJ], sn[QJ];
  int32_t idx[QJ];
#pragma unroll
  for (int q = 0; q < QJ; ++q) {
    c1[q] = ctab[j[q]];
    s1[q] = tab[j[q]];
    cs[q] = 1.f;
    sn[q] = 0.f;
    idx[q] = 0;
#pragma unroll
    for (int s = 0; s < SG; ++s) acc[q][s] = 0.f;
  }
  for (int32_t i = 0; i < m; ++i) {
#pragma unroll
    for (int q = 0; q < QJ; ++q) {
      idx[q] += j[q];
      if (idx[q] >= P) idx[q] -= P;
      if ((i & 31) == 0) {
        cs[q] = ctab[idx[q]];
        sn[q] = tab[idx[q]];
      } else {
        const float c = cs[q] * c1[q] - sn[q] * s1[q];
        sn[q] = fmaf(sn[q], c1[q], cs[q] * s1[q]);
        cs[q] = c;
      }
    }
    const float4* row = reinterpret_cast<const float4*>(src + (size_t)i * SG);
#pragma unroll
    for (int p = 0; p < SG / 4; ++p) {
      const float4 v = row[p];
#pragma unroll
      for (int q = 0; q < QJ; ++q) {
        acc[q][4 * p + 0] = fmaf(sn[q], v.x, acc[q][4 * p + 0]);
        acc[q][4 * p + 1] = fmaf(sn[q], v.y, acc[q][4 * p + 1]);
        acc[q][4 * p + 2] = fmaf(sn[q], v.z, acc[q][4 * p + 2]);
        acc[q][4 * p + 3] = fmaf(sn[q], v.w, acc[q][4 * p + 3]);
      }
    }
  }
}

// Rows [m][SG] of a sample-minor array (row stride S, first sample s0, kv valid
// samples) into shared memory, zero-padded to SG: float4 loads with several in
// flight per thread when the rows are 16-byte aligned and whole.
template <int SG>
__device__ __forceinline__ void stage_rows(const float* __restrict__ src, int64_t S, int kv,
                                           int32_t m, float* dst) {
  if (kv == SG && (S & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    constexpr int Q = SG / 4;  // float4 per row
    const int32_t total = m * Q;
    int32_t t = threadIdx.x;
    for (; t + 3 * (int32_t)blockDim.x < total; t += 4 * blockDim.x) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int32_t tt = t + u * blockDim.x;
        v[u] = *reinterpret_cast<const float4*>(src + (int64_t)(tt / Q) * S + 4 * (tt % Q));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) reinterpret_cast<float4*>(dst)[t + u * blockDim.x] = v[u];
    }
    for (; t < total; t += blockDim.x)
      reinterpret_cast<float4*>(dst)[t] =
          *reinterpret_cast<const float4*>(src + (int64_t)(t / Q) * S + 4 * (t % Q));
  } else {
    for (int32_t t = threadIdx.x; t < m * SG; t += blockDim.x) {
      const int32_t i = t / SG, c = t - i * SG;
      dst[t] = c < kv ? src[(int64_t)i * S + c] : 0.f;
    }
  }
}

// a[s] += r * row[s]
template <int SG>
__device__ __forceinline__ void spec_acc(float r, const float* rowp, float (&a)[SG]) {
  const float4* row = reinterpret_cast<const float4*>(rowp);
#pragma unroll
  for (int q = 0; q < SG / 4; ++q) {
    const float4 v = row[q];
    a[4 * q + 0] = fmaf(r, v.x, a[4 * q + 0]);
    a[4 * q + 1] = fmaf(r, v.y, a[4 * q + 1]);
    a[4 * q + 2] = fmaf(r, v.z, a[4 * q + 2]);
    a[4 * q + 3] = fmaf(r, v.w, a[4 * q + 3]);
  }
}

// a[s] += r * row[s], b[s] += t * row[s]
template <int SG>
__device__ __forceinline__ void spec_acc2(float r, float t, const float* rowp, float (&a)[SG],
                                          float (&b)[SG]) {
  const float4* row = reinterpret_cast<const float4*>(rowp);
#pragma unroll
  for (int q = 0; q < SG / 4; ++q) {
    const float4 v = row[q];
    a[4 * q + 0] = fmaf(r, v.x, a[4 * q + 0]);
    a[4 * q + 1] = fmaf(r, v.y, a[4 * q + 1]);
    a[4 * q + 2] = fmaf(r, v.z, a[4 * q + 2]);
    a[4 * q + 3] = fmaf(r, v.w, a[4 * q + 3]);
    b[4 * q + 0] = fmaf(t, v.x, b[4 * q + 0]);
    b[4 * q + 1] = fmaf(t, v.y, b[4 * q + 1]);
    b[4 * q + 2] = fmaf(t, v.z, b[4 * q + 2]);
    b[4 * q + 3] = fmaf(t, v.w, b[4 * q + 3]);
  }
}

template <int SG>
__host__ __device__ constexpr size_t spec_condense_floats(int32_t mmax) {
  return 4 * ((size_t)mmax + 1) + (size_t)mmax + 2 * (size_t)mmax * SG + 4;
}

// Forward transform of the edge's noise (written to bhat, rows like b) and
// the two end values of T_l^-1 b_I for every node, added into gvec.
template <int SG, int QJ>
__global__ void __launch_bounds__(256)
    spec_condense_kernel(DevGraph g, DevNodes nd, double kappa2, int64_t S,
                         const float* __restrict__ b, const int32_t* __restrict__ edges,
                         int32_t n_edges, int32_t mmax, float* __restrict__ bhat,
                         double* __restrict__ gvec) {
  extern __shared__ __align__(16) float spec_sm[];
  float* bs = spec_sm;                          // [mmax][SG] noise rows
  float* bt = bs + (size_t)mmax * SG;           // [mmax][SG] phi_j bh_j
  float* tab = bt + (size_t)mmax * SG;          // [2 (mmax + 1)] sin
  float* ctab = tab + 2 * ((size_t)mmax + 1);   // [2 (mmax + 1)] cos
  float* sig = ctab + 2 * ((size_t)mmax + 1);   // [mmax]
  const int64_t nsg = (S + SG - 1) / SG;
  const int64_t units = (int64_t)n_edges * nsg;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int32_t e = edges[u / nsg];
    const int64_t s0 = (u % nsg) * SG;
    const int32_t m = g.nel[e] - 1;  // 1 <= m <= mmax for binned edges
    const int64_t off = g.ioff[e];
    const int kv = (int)(S - s0 < SG ? S - s0 : SG);
    __syncthreads();  // the previous unit is done with the shared arrays
    spec_tables(m, tab, ctab, sig);
    stage_rows<SG>(b + (g.nv + off) * S + s0, S, kv, m, bs);
    __syncthreads();
    const float scale = sqrtf(2.f / (float)(m + 1));
    // forward transform: modes t + q blockDim (q < QJ) per thread share every
    // row load; the bin's QJ blockDim >= m, so one pass covers the edge
    for (int32_t jb = 0; jb < m; jb += QJ * blockDim.x) {
      int32_t jj[QJ];
#pragma unroll
      for (int q = 0; q < QJ; ++q) {
        const int32_t j = jb + q * blockDim.x + threadIdx.x;
        jj[q] = j < m ? j + 1 : 0;
      }
      if (jj[0] == 0) continue;
      float acc[QJ][SG];
      dst_rows<SG, QJ>(m, jj, tab, ctab, bs, acc);
#pragma unroll
      for (int q = 0; q < QJ; ++q) {
        if (jj[q] == 0) continue;
        const int32_t j = jj[q] - 1;
        const float phi = scale * tab[j + 1];
        float* bo = bhat + (off + j) * S + s0;
#pragma unroll
        for (int s = 0; s < SG; ++s) {
          const float bh = scale * acc[q][s];
          if (s < kv) bo[s] = bh;
          bt[(size_t)j * SG + s] = phi * bh;
        }
      }
    }
    __syncthreads();
    const double h = g.he[e];
    const float h2f = (float)(h * h);
    const int32_t va = g.eu[e], vb = g.ev[e];
    // end values: two nodes per thread share every row load
    for (int32_t l0 = 2 * threadIdx.x; l0 < nd.L; l0 += 2 * blockDim.x) {
      const bool two = l0 + 1 < nd.L;
      const float dl0 = nd.shift[l0] * h2f;
      const float dl1 = two ? nd.shift[l0 + 1] * h2f : 1.f;
      float od[2][SG], ev[2][SG];
#pragma unroll
      for (int s = 0; s < SG; ++s) od[0][s] = ev[0][s] = od[1][s] = ev[1][s] = 0.f;
      // modes j + 1 in pairs: odd mode (j even) into od, even mode into ev
      for (int32_t j = 0; j < m; j += 2) {
        spec_acc2<SG>(__fdividef(1.f, dl0 + sig[j]), __fdividef(1.f, dl1 + sig[j]),
                      bt + (size_t)j * SG, od[0], od[1]);
        if (j + 1 < m)
          spec_acc2<SG>(__fdividef(1.f, dl0 + sig[j + 1]), __fdividef(1.f, dl1 + sig[j + 1]),
                        bt + (size_t)(j + 1) * SG, ev[0], ev[1]);
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (q == 1 && !two) break;
        double* gl = gvec + ((int64_t)(l0 + q) * S + s0) * g.nv;
#pragma unroll
        for (int s = 0; s < SG; ++s) {
          if (s < kv) {
            atomicAdd(gl + (int64_t)s * g.nv + va, (double)(od[q][s] + ev[q][s]));
            atomicAdd(gl + (int64_t)s * g.nv + vb, (double)(od[q][s] - ev[q][s]));
          }
        }
      }
    }
  }
}

template <int SG>
__host__ __device__ constexpr size_t spec_recover_floats(int32_t mmax) {
  return (size_t)mmax * SG + 4 * ((size_t)mmax + 1) + (size_t)mmax +
         (size_t)kSpecLChunk * (2 + 2 * SG) + 4;
}

// U_I = Phi c with c from bhat and the weighted vertex values xw[l][v][s] = w_l u_v^(l).
template <int SG, int QJ, typename OutT>
__global__ void __launch_bounds__(256)
    spec_recover_kernel(DevGraph g, DevNodes nd, double kappa2, int64_t S,
                        const int32_t* __restrict__ edges, int32_t n_edges, int32_t mmax,
                        const float* __restrict__ bhat, const float* __restrict__ xw,
                        OutT* __restrict__ out) {
  extern __shared__ __align__(16) float spec_sm[];
  float* cs = spec_sm;                            // [mmax][SG] bh, then c
  float* xp = cs + (size_t)mmax * SG;             // [chunk][SG] xa + xb
  float* xm = xp + (size_t)kSpecLChunk * SG;      // [chunk][SG] xa - xb
  float* dls = xm + (size_t)kSpecLChunk * SG;     // [chunk] delta_l
  float* scs = dls + kSpecLChunk;                 // [chunk] sc_l
  float* tab = scs + kSpecLChunk;                 // [2 (mmax + 1)] sin
  float* ctab = tab + 2 * ((size_t)mmax + 1);     // [2 (mmax + 1)] cos
  float* sig = ctab + 2 * ((size_t)mmax + 1);     // [mmax]
  const int64_t nsg = (S + SG - 1) / SG;
  const int64_t units = (int64_t)n_edges * nsg;
  constexpr int kJ = QJ;  // modes per thread held in registers (pass over l shared)
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int32_t e = edges[u / nsg];
    const int64_t s0 = (u % nsg) * SG;
    const int32_t m = g.nel[e] - 1;
    const int64_t off = g.ioff[e];
    const int kv = (int)(S - s0 < SG ? S - s0 : SG);
    const double h = g.he[e];
    const float hf = (float)h, h2f = (float)(h * h);
    const int32_t va = g.eu[e], vb = g.ev[e];
    __syncthreads();
    spec_tables(m, tab, ctab, sig);
    stage_rows<SG>(bhat + off * S + s0, S, kv, m, cs);
    const float scale = sqrtf(2.f / (float)(m + 1));
    // modes j0 + kJ * blockDim * pass ...: each thread owns up to kJ modes per pass
    for (int32_t jb = 0; jb < m; jb += kJ * blockDim.x) {
      float C[kJ][SG], D[kJ];
#pragma unroll
      for (int q = 0; q < kJ; ++q) {
        D[q] = 0.f;
#pragma unroll
        for (int s = 0; s < SG; ++s) C[q][s] = 0.f;
      }
      for (int32_t l0 = 0; l0 < nd.L; l0 += kSpecLChunk) {
        const int32_t lc = nd.L - l0 < kSpecLChunk ? nd.L - l0 : kSpecLChunk;
        __syncthreads();  // tables and cs visible; previous chunk consumed
        for (int32_t t = threadIdx.x; t < lc; t += blockDim.x) {
          const int32_t l = l0 + t;
          dls[t] = nd.shift[l] * h2f;
          scs[t] = nd.wgam[l] * hf;
        }
        // the two ends' rows xw[l][v][s0 .. s0 + SG) (contiguous per node)
        for (int32_t t = threadIdx.x; t < lc * SG; t += blockDim.x) {
          const int32_t lq = t / SG, s = t - lq * SG;
          float a = 0.f, c = 0.f;
          if (s < kv) {
            const int64_t l = l0 + lq;
            a = xw[(l * g.nv + va) * S + s0 + s];
            c = xw[(l * g.nv + vb) * S + s0 + s];
          }
          xp[t] = a + c;
          xm[t] = a - c;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kJ; ++q) {
          const int32_t j = jb + q * blockDim.x + threadIdx.x;  // 0-based mode index
          if (j < m) {
            const float sj = sig[j];
            const float* X = (j & 1) ? xm : xp;  // mode j + 1 odd <=> j even
            for (int32_t lq = 0; lq < lc; ++lq) {
              const float r = __fdividef(1.f, dls[lq] + sj);
              D[q] = fmaf(scs[lq], r, D[q]);
              spec_acc<SG>(r, X + (size_t)lq * SG, C[q]);
            }
          }
        }
      }
      // c_j = D_j bh_j + phi_j C_j, in place over the thread's own rows
#pragma unroll
      for (int q = 0; q < kJ; ++q) {
        const int32_t j = jb + q * blockDim.x + threadIdx.x;
        if (j < m) {
          const float phi = scale * tab[j + 1];
#pragma unroll
          for (int s = 0; s < SG; ++s)
            cs[(size_t)j * SG + s] = fmaf(D[q], cs[(size_t)j * SG + s], phi * C[q][s]);
        }
      }
    }
    __syncthreads();
    // inverse transform: output nodes t + q blockDim (q < QJ) per thread
    for (int32_t ib = 0; ib < m; ib += QJ * blockDim.x) {
      int32_t ii[QJ];
#pragma unroll
      for (int q = 0; q < QJ; ++q) {
        const int32_t i = ib + q * blockDim.x + threadIdx.x;
        ii[q] = i < m ? i + 1 : 0;
      }
      if (ii[0] == 0) continue;
      float acc[QJ][SG];
      dst_rows<SG, QJ>(m, ii, tab, ctab, cs, acc);
#pragma unroll
      for (int q = 0; q < QJ; ++q) {
        if (ii[q] == 0) continue;
        OutT* o = out + (int64_t)s0 * g.n + g.nv + off + ii[q] - 1;
#pragma unroll
        for (int s = 0; s < SG; ++s)
          if (s < kv) o[(int64_t)s * g.n] = (OutT)(scale * acc[q][s]);
      }
    }
  }
}

__global__ void node_consts_kernel(DevNodes nd, double kappa2, float* __restrict__ shift,
                                   float* __restrict__ wgam) {
  for (int32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < nd.L; l += gridDim.x * blockDim.x) {
    const double gam = nd.gamma[l];
    shift[l] = (float)(nd.alpha[l] / gam + kappa2);
    wgam[l] = (float)(nd.weight[l] / gam);
  }
}

int grid_units(int64_t units) {
  int64_t b = units < sm_count() * 16 ? units : sm_count() * 16;
  return b < 1 ? 1 : (int)b;
}

// The two halves around the tensor-core transforms (dst_gemm.cu): they only
// contract bhat with 1 / mu_jl, so one node (ends) or one mode (coefficients)
// per thread and a shared-memory footprint of one edge's rows keep several
// CTAs per SM.
}  // namespace

// Spectral bins: interior-node limit, threads per CTA and modes per thread
// (threads x modes >= limit: one pass over the edge per transform).
struct SpecBin {
  int32_t mmax, threads, qj;
};
constexpr SpecBin kSpecBins[] = {{64, 128, 1},  {128, 128, 1}, {256, 128, 2}, {384, 128, 3},
                                 {512, 128, 4}, {768, 256, 3}, {1024, 256, 4}};
constexpr int kNumSpecBins = sizeof(kSpecBins) / sizeof(kSpecBins[0]);

void launch_node_consts(const DevNodes& nd, double kappa2, float* shift, float* wgam,
                        cudaStream_t st) {
  int blocks = (nd.L + 255) / 256;
  if (blocks > sm_count()) blocks = sm_count();
  node_consts_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(nd, kappa2, shift, wgam);
}

int spec_bins(int32_t* mmax) {
  for (int i = 0; i < kNumSpecBins; ++i) mmax[i] = kSpecBins[i].mmax;
  return kNumSpecBins;
}

template <int QJ>
void spec_condense_bin(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S,
                       const float* b, const int32_t* e, int32_t n, const SpecBin& bin,
                       float* bhat, double* gvec, cudaStream_t st) {
  const size_t smem = spec_condense_floats<kSpecSG>(bin.mmax) * sizeof(float);
  cudaFuncSetAttribute(spec_condense_kernel<kSpecSG, QJ>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t units = (int64_t)n * ((S + kSpecSG - 1) / kSpecSG);
  spec_condense_kernel<kSpecSG, QJ><<<grid_units(units), bin.threads, smem, st>>>(
      g, nd, kappa2, S, b, e, n, bin.mmax, bhat, gvec);
}

int launch_spec_condense(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S,
                         const float* b, const int32_t* bin_edges, const int32_t* bin_count,
                         float* bhat, double* gvec, cudaStream_t st) {
  const int32_t* e = bin_edges;
  int launches = 0;
  for (int i = 0; i < kNumSpecBins; ++i) {
    const int32_t n = bin_count[i];
    if (n > 0) {
      const SpecBin& bn = kSpecBins[i];
      switch (bn.qj) {
        case 1: spec_condense_bin<1>(g, nd, kappa2, S, b, e, n, bn, bhat, gvec, st); break;
        case 2: spec_condense_bin<2>(g, nd, kappa2, S, b, e, n, bn, bhat, gvec, st); break;
        case 3: spec_condense_bin<3>(g, nd, kappa2, S, b, e, n, bn, bhat, gvec, st); break;
        default: spec_condense_bin<4>(g, nd, kappa2, S, b, e, n, bn, bhat, gvec, st); break;
      }
      ++launches;
    }
    e += n;
  }
  return launches;
}

template <int QJ, typename OutT>
void spec_recover_bin(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S,
                      const int32_t* e, int32_t n, const SpecBin& bin, const float* bhat,
                      const float* xw, OutT* out, cudaStream_t st) {
  const size_t smem = spec_recover_floats<kSpecSG>(bin.mmax) * sizeof(float);
  cudaFuncSetAttribute(spec_recover_kernel<kSpecSG, QJ, OutT>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t units = (int64_t)n * ((S + kSpecSG - 1) / kSpecSG);
  spec_recover_kernel<kSpecSG, QJ, OutT><<<grid_units(units), bin.threads, smem, st>>>(
      g, nd, kappa2, S, e, n, bin.mmax, bhat, xw, out);
}

template <typename OutT>
int launch_spec_recover(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S,
                        const int32_t* bin_edges, const int32_t* bin_count, const float* bhat,
                        const float* xw, OutT* out, cudaStream_t st) {
  const int32_t* e = bin_edges;
  int launches = 0;
  for (int i = 0; i < kNumSpecBins; ++i) {
    const int32_t n = bin_count[i];
    if (n > 0) {
      const SpecBin& bn = kSpecBins[i];
      switch (bn.qj) {
        case 1: spec_recover_bin<1, OutT>(g, nd, kappa2, S, e, n, bn, bhat, xw, out, st); break;
        case 2: spec_recover_bin<2, OutT>(g, nd, kappa2, S, e, n, bn, bhat, xw, out, st); break;
        case 3: spec_recover_bin<3, OutT>(g, nd, kappa2, S, e, n, bn, bhat, xw, out, st); break;
        default: spec_recover_bin<4, OutT>(g, nd, kappa2, S, e, n, bn, bhat, xw, out, st); break;
      }
      ++launches;
    }
    e += n;
  }
  return launches;
}
template int launch_spec_recover<float>(const DevGraph&, const DevNodes&, double, int64_t,
                                        const int32_t*, const int32_t*, const float*,
                                        const float*, float*, cudaStream_t);
template int launch_spec_recover<double>(const DevGraph&, const DevNodes&, double, int64_t,
                                         const int32_t*, const int32_t*, const float*,
                                         const float*, double*, cudaStream_t);

}  // namespace grf
