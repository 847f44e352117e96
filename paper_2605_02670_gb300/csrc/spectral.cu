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

constexpr int kSpecThreads = 128;
constexpr int kSpecLChunk = 128;  // nodes staged per pass in the recovery

// sin(pi k / (m+1)) for k < 2(m+1) (argument reduced to [0, 1/2] before
// rounding), the mode shifts sig_j = 4 sin^2(pi j / (2(m+1))), j = 1..m.
__device__ __forceinline__ void spec_tables(int32_t m, float* tab, float* sig) {
  const int32_t P = 2 * (m + 1);
  for (int32_t k = threadIdx.x; k < P; k += blockDim.x) {
    int32_t kk = k < m + 1 ? k : k - (m + 1);  // sin(pi (k - (m+1)) / (m+1)) = -sin(...)
    const float sgn = k < m + 1 ? 1.f : -1.f;
    kk = kk <= (m + 1) / 2 ? kk : (m + 1) - kk;  // sin(pi x) = sin(pi (1 - x))
    tab[k] = sgn * sinpif((float)kk / (float)(m + 1));
  }
  for (int32_t j = threadIdx.x; j < m; j += blockDim.x) {
    const float sh = 2.f * sinpif((float)(j + 1) / (float)(2 * (m + 1)));
    sig[j] = sh * sh;
  }
}

// acc[s] = sum_{i=1..m} sin(pi i j / (m+1)) src[i-1][s]   (table index i j mod P)
template <int SG>
__device__ __forceinline__ void dst_row(int32_t m, int32_t j, const float* tab,
                                        const float* src, float (&acc)[SG]) {
  const int32_t P = 2 * (m + 1);
#pragma unroll
  for (int s = 0; s < SG; ++s) acc[s] = 0.f;
  int32_t idx = 0;
  for (int32_t i = 0; i < m; ++i) {
    idx += j;
    if (idx >= P) idx -= P;
    const float f = tab[idx];
    const float4* row = reinterpret_cast<const float4*>(src + (size_t)i * SG);
#pragma unroll
    for (int q = 0; q < SG / 4; ++q) {
      const float4 v = row[q];
      acc[4 * q + 0] = fmaf(f, v.x, acc[4 * q + 0]);
      acc[4 * q + 1] = fmaf(f, v.y, acc[4 * q + 1]);
      acc[4 * q + 2] = fmaf(f, v.z, acc[4 * q + 2]);
      acc[4 * q + 3] = fmaf(f, v.w, acc[4 * q + 3]);
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

template <int SG>
__host__ __device__ constexpr size_t spec_condense_floats(int32_t mmax) {
  return 2 * ((size_t)mmax + 1) + (size_t)mmax + 2 * (size_t)mmax * SG + 4;
}

// Forward transform of the edge's noise (written to bhat, rows like b) and
// the two end values of T_l^-1 b_I for every node, added into gvec.
template <int SG>
__global__ void __launch_bounds__(kSpecThreads)
    spec_condense_kernel(DevGraph g, DevNodes nd, double kappa2, int64_t S,
                         const float* __restrict__ b, const int32_t* __restrict__ edges,
                         int32_t n_edges, int32_t mmax, float* __restrict__ bhat,
                         double* __restrict__ gvec) {
  extern __shared__ __align__(16) float spec_sm[];
  float* bs = spec_sm;                          // [mmax][SG] noise rows
  float* bt = bs + (size_t)mmax * SG;           // [mmax][SG] phi_j bh_j
  float* tab = bt + (size_t)mmax * SG;          // [2 (mmax + 1)]
  float* sig = tab + 2 * ((size_t)mmax + 1);    // [mmax]
  const int64_t nsg = (S + SG - 1) / SG;
  const int64_t units = (int64_t)n_edges * nsg;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int32_t e = edges[u / nsg];
    const int64_t s0 = (u % nsg) * SG;
    const int32_t m = g.nel[e] - 1;  // 1 <= m <= mmax for binned edges
    const int64_t off = g.ioff[e];
    const int kv = (int)(S - s0 < SG ? S - s0 : SG);
    __syncthreads();  // the previous unit is done with the shared arrays
    spec_tables(m, tab, sig);
    const float* bI = b + (g.nv + off) * S + s0;
    for (int32_t t = threadIdx.x; t < m * SG; t += blockDim.x) {
      const int32_t i = t / SG, s = t - i * SG;
      bs[t] = s < kv ? bI[(int64_t)i * S + s] : 0.f;
    }
    __syncthreads();
    const float scale = sqrtf(2.f / (float)(m + 1));
    for (int32_t j = threadIdx.x; j < m; j += blockDim.x) {
      float acc[SG];
      dst_row<SG>(m, j + 1, tab, bs, acc);
      const float phi = scale * tab[j + 1];
      float* bo = bhat + (off + j) * S + s0;
#pragma unroll
      for (int s = 0; s < SG; ++s) {
        const float bh = scale * acc[s];
        if (s < kv) bo[s] = bh;
        bt[(size_t)j * SG + s] = phi * bh;
      }
    }
    __syncthreads();
    const double h = g.he[e];
    const int32_t va = g.eu[e], vb = g.ev[e];
    for (int32_t l = threadIdx.x; l < nd.L; l += blockDim.x) {
      const float dl = (float)((nd.alpha[l] / nd.gamma[l] + kappa2) * h * h);
      float od[SG], ev[SG];
#pragma unroll
      for (int s = 0; s < SG; ++s) od[s] = ev[s] = 0.f;
      // modes j + 1 in pairs: odd mode (j even) into od, even mode into ev
      for (int32_t j = 0; j < m; j += 2) {
        spec_acc<SG>(__fdividef(1.f, dl + sig[j]), bt + (size_t)j * SG, od);
        if (j + 1 < m) spec_acc<SG>(__fdividef(1.f, dl + sig[j + 1]), bt + (size_t)(j + 1) * SG, ev);
      }
      double* gl = gvec + ((int64_t)l * S + s0) * g.nv;
#pragma unroll
      for (int s = 0; s < SG; ++s) {
        if (s < kv) {
          atomicAdd(gl + (int64_t)s * g.nv + va, (double)(od[s] + ev[s]));
          atomicAdd(gl + (int64_t)s * g.nv + vb, (double)(od[s] - ev[s]));
        }
      }
    }
  }
}

template <int SG>
__host__ __device__ constexpr size_t spec_recover_floats(int32_t mmax) {
  return (size_t)mmax * SG + 2 * ((size_t)mmax + 1) + (size_t)mmax +
         (size_t)kSpecLChunk * (2 + 2 * SG) + 4;
}

// U_I = Phi c with c from bhat and the weighted vertex values xw = w_l u_v^(l).
template <int SG, typename OutT>
__global__ void __launch_bounds__(kSpecThreads)
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
  float* tab = scs + kSpecLChunk;                 // [2 (mmax + 1)]
  float* sig = tab + 2 * ((size_t)mmax + 1);      // [mmax]
  const int64_t nsg = (S + SG - 1) / SG;
  const int64_t units = (int64_t)n_edges * nsg;
  constexpr int kJ = 2;  // modes per thread held in registers (pass over l shared)
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int32_t e = edges[u / nsg];
    const int64_t s0 = (u % nsg) * SG;
    const int32_t m = g.nel[e] - 1;
    const int64_t off = g.ioff[e];
    const int kv = (int)(S - s0 < SG ? S - s0 : SG);
    const double h = g.he[e];
    const int32_t va = g.eu[e], vb = g.ev[e];
    __syncthreads();
    spec_tables(m, tab, sig);
    const float* bh = bhat + off * S + s0;
    for (int32_t t = threadIdx.x; t < m * SG; t += blockDim.x) {
      const int32_t i = t / SG, s = t - i * SG;
      cs[t] = s < kv ? bh[(int64_t)i * S + s] : 0.f;
    }
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
          const double gam = nd.gamma[l];
          dls[t] = (float)((nd.alpha[l] / gam + kappa2) * h * h);
          scs[t] = (float)(nd.weight[l] * h / gam);
        }
        for (int32_t t = threadIdx.x; t < lc * SG; t += blockDim.x) {
          const int32_t lq = t / SG, s = t - lq * SG;
          float a = 0.f, c = 0.f;
          if (s < kv) {
            const int64_t base = ((int64_t)(l0 + lq) * S + s0 + s) * g.nv;
            a = xw[base + va];
            c = xw[base + vb];
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
    for (int32_t i = threadIdx.x; i < m; i += blockDim.x) {
      float acc[SG];
      dst_row<SG>(m, i + 1, tab, cs, acc);
      OutT* o = out + (int64_t)s0 * g.n + g.nv + off + i;
#pragma unroll
      for (int s = 0; s < SG; ++s)
        if (s < kv) o[(int64_t)s * g.n] = (OutT)(scale * acc[s]);
    }
  }
}

int grid_units(int64_t units) {
  int64_t b = units < 152 * 16 ? units : 152 * 16;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

int spec_bins(int32_t* mmax) {
  static const int32_t mm[] = {32, 64, 128, 256, 512, 1024};
  for (int i = 0; i < 6; ++i) mmax[i] = mm[i];
  return 6;
}

int launch_spec_condense(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S,
                         const float* b, const int32_t* bin_edges, const int32_t* bin_count,
                         float* bhat, double* gvec, cudaStream_t st) {
  int32_t mm[kMaxBins];
  const int nb = spec_bins(mm);
  const int32_t* e = bin_edges;
  int launches = 0;
  for (int i = 0; i < nb; ++i) {
    const int32_t n = bin_count[i];
    if (n > 0) {
      const size_t smem = spec_condense_floats<kSpecSG>(mm[i]) * sizeof(float);
      cudaFuncSetAttribute(spec_condense_kernel<kSpecSG>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      const int64_t units = (int64_t)n * ((S + kSpecSG - 1) / kSpecSG);
      spec_condense_kernel<kSpecSG><<<grid_units(units), kSpecThreads, smem, st>>>(
          g, nd, kappa2, S, b, e, n, mm[i], bhat, gvec);
      ++launches;
    }
    e += n;
  }
  return launches;
}

template <typename OutT>
int launch_spec_recover(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S,
                        const int32_t* bin_edges, const int32_t* bin_count, const float* bhat,
                        const float* xw, OutT* out, cudaStream_t st) {
  int32_t mm[kMaxBins];
  const int nb = spec_bins(mm);
  const int32_t* e = bin_edges;
  int launches = 0;
  for (int i = 0; i < nb; ++i) {
    const int32_t n = bin_count[i];
    if (n > 0) {
      const size_t smem = spec_recover_floats<kSpecSG>(mm[i]) * sizeof(float);
      cudaFuncSetAttribute(spec_recover_kernel<kSpecSG, OutT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      const int64_t units = (int64_t)n * ((S + kSpecSG - 1) / kSpecSG);
      spec_recover_kernel<kSpecSG, OutT><<<grid_units(units), kSpecThreads, smem, st>>>(
          g, nd, kappa2, S, e, n, mm[i], bhat, xw, out);
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
