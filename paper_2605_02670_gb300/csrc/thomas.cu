// Edge-interior sweeps of the domain decomposition (Sec. 3, Phases 3 and 5).
//
// On edge e the interior block of A_l = alpha_l M_L + gamma_l K is c T with
// c = gamma_l / h_e and T = tridiag(-1, 2 + delta, -1), delta =
// (alpha_l / gamma_l + kappa^2) h_e^2. Thomas elimination of T (Eq.
// thomas_coefficients) has pivots p_i = 1 + q_i with the excess recurrence
//   q_1 = 1 + delta,  q_{i+1} = delta + q_i / (1 + q_i),
// which never subtracts, so it keeps full relative accuracy of delta even in
// FP32 where 2 + delta would round delta away. Forward substitution is
// y_i = r_i + y_{i-1} / p_{i-1}, back substitution x_i = (y_i + x_{i+1}) / p_i.
//
// condense: g_v = b_v + sum_{e at v} (T^{-1} b_I^(e))_{node next to v}
//   (Eq. local_reduced_schur: -A_vI A_II^{-1} = c T^{-1} / c). The end value
//   next to edge_v is one forward elimination from edge_u's side; by symmetry
//   of the constant-coefficient T the end value next to edge_u is the same
//   elimination run from edge_v's side. Both run in one pass over b_I.
// recover: U_I = sum_l w_l T^{-1} (b_I / c + u_a e_1 + u_b e_m) (Eq.
//   internal_recovery) with the quadrature sum (Phase 5) fused: the weight is
//   folded into the right-hand side and the sum over nodes is kept in FP64.
#include <type_traits>

#include "grf_internal.h"

namespace grf {
namespace {

constexpr int kSG = 4;  // samples per thread: pivots are shared across them

int grid_for(int64_t total, int threads) {
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > sm_count() * 64) blocks = sm_count() * 64;
  return blocks < 1 ? 1 : (int)blocks;
}

template <typename T>
__global__ void gvec_init_kernel(DevGraph g, int32_t L, int64_t S, const T* __restrict__ b,
                                 double* __restrict__ gvec) {
  const int64_t total = (int64_t)L * S * g.nv;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t % g.nv;
    const int64_t s = (t / g.nv) % S;
    gvec[t] = (double)b[v * S + s];
  }
}

// Reciprocal of a pivot. FP32: the SFU approximation (relative error a few
// 1e-8); the sweeps contract, so pivot errors of that size stay at that size.
__device__ __forceinline__ float rcp_piv(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_piv(double x) { return 1.0 / x; }

// q_K = delta / 2 + sinh(theta) coth(K theta) reaches q* = delta / 2 + sinh(theta)
// in the working precision once 2 exp(-2 K theta) is below half an ulp:
// K theta >= 9 in FP32, >= 19 in FP64. First node index from which q_K = q*
// (clamped to [2, m + 1]).
template <typename T>
__device__ __forceinline__ int32_t converged_from(T delta, int32_t m) {
  constexpr T kTheta = sizeof(T) == 4 ? (T)9 : (T)19;
  const T th = (T)2 * asinh((T)0.5 * sqrt(delta));
  const T k = th > (T)0 ? ceil(kTheta / th) : (T)(m + 1);
  if (!(k < (T)(m + 1))) return m + 1;
  return k < (T)2 ? 2 : (int32_t)k;
}

// One CTA per (edge, group of kSG samples): the edge's noise rows are staged in
// shared memory once ([m][kSG]) and every thread runs the two end eliminations
// of one quadrature node from there (all threads read the same row at the same
// step: broadcast). The pivot recurrence of a node is shared by its kSG samples
// and runs only until it has converged; from there on the pivot is the fixed
// point 1 + q*.
// The two end eliminations of one node over rows src[i * stride .. + kSG).
// Only the first kv (<= kSG) samples of a row are read; kStaged: rows are
// contiguous in shared memory (stride kSG, all kSG samples), read as vectors.
template <typename T, bool kStaged>
__device__ __forceinline__ void load_row(const T* p, int kv, T (&v)[kSG]) {
  if constexpr (kStaged && std::is_same<T, float>::value) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (kStaged) {
    const double2 t0 = *reinterpret_cast<const double2*>(p);
    const double2 t1 = *reinterpret_cast<const double2*>(p + 2);
    v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
  } else {
#pragma unroll
    for (int k = 0; k < kSG; ++k) v[k] = k < kv ? p[k] : (T)0;
  }
}

template <typename T, bool kStaged>
__device__ __forceinline__ void end_sweeps(const T* src, int64_t stride, int32_t m, T delta,
                                           int kv, T (&yf)[kSG], T (&yr)[kSG], T& rp_out) {
  load_row<T, kStaged>(src, kv, yf);
  load_row<T, kStaged>(src + (int64_t)(m - 1) * stride, kv, yr);
  T q = (T)1 + delta;
  T rp = rcp_piv((T)1 + q);
  const int32_t kc = converged_from<T>(delta, m);  // nodes >= kc have q = q*
  int32_t i = 1;
  for (; i < kc && i < m; ++i) {
    T rf[kSG], rr[kSG];
    load_row<T, kStaged>(src + (int64_t)i * stride, kv, rf);
    load_row<T, kStaged>(src + (int64_t)(m - 1 - i) * stride, kv, rr);
#pragma unroll
    for (int k = 0; k < kSG; ++k) {
      yf[k] = rf[k] + rp * yf[k];
      yr[k] = rr[k] + rp * yr[k];
    }
    q = delta + q * rp;
    rp = rcp_piv((T)1 + q);
  }
  if (i < m) {
    rp = rcp_piv((T)1 + (T)0.5 * delta + sqrt(delta * ((T)1 + (T)0.25 * delta)));
#pragma unroll 4
    for (; i < m; ++i) {
      T rf[kSG], rr[kSG];
      load_row<T, kStaged>(src + (int64_t)i * stride, kv, rf);
      load_row<T, kStaged>(src + (int64_t)(m - 1 - i) * stride, kv, rr);
#pragma unroll
      for (int k = 0; k < kSG; ++k) {
        yf[k] = rf[k] + rp * yf[k];
        yr[k] = rr[k] + rp * yr[k];
      }
    }
  }
  rp_out = rp;
}

// Edges with more than stage_max interior nodes read their rows from global
// memory instead of shared memory.
// edges (may be null: every edge) lists the n_edges edges to process.
template <typename T>
__global__ void __launch_bounds__(256) condense_kernel(DevGraph g, DevNodes nd, double kappa2,
                                                      int64_t S, const T* __restrict__ b,
                                                      double* __restrict__ gvec,
                                                      int32_t stage_max,
                                                      const int32_t* __restrict__ edges,
                                                      int32_t n_edges) {
  extern __shared__ __align__(16) unsigned char cond_sm[];
  T* sb = reinterpret_cast<T*>(cond_sm);
  const int64_t nsg = (S + kSG - 1) / kSG;
  const int64_t units = (int64_t)n_edges * nsg;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int32_t e = edges ? edges[u / nsg] : (int32_t)(u / nsg);
    const int64_t s0 = (u % nsg) * kSG;
    const int32_t m = g.nel[e] - 1;
    if (m <= 0) continue;  // uniform across the CTA
    const bool staged = m <= stage_max;
    const int kv = (int)(S - s0 < kSG ? S - s0 : kSG);
    const T* bI = b + (g.nv + g.ioff[e]) * S;
    if (staged) {
      __syncthreads();  // the previous unit is done with sb
      for (int32_t i = threadIdx.x; i < m * kSG; i += blockDim.x) {
        const int32_t row = i / kSG, k = i - row * kSG;
        sb[i] = s0 + k < S ? bI[(int64_t)row * S + s0 + k] : (T)0;
      }
      __syncthreads();
    }
    const double h = g.he[e];
    const int32_t a = g.eu[e], bv = g.ev[e];
    for (int32_t l = threadIdx.x; l < nd.L; l += blockDim.x) {
      const T delta = (T)((nd.alpha[l] / nd.gamma[l] + kappa2) * h * h);
      T yf[kSG], yr[kSG], rp;
      if (staged)
        end_sweeps<T, true>(sb, kSG, m, delta, kSG, yf, yr, rp);
      else
        end_sweeps<T, false>(bI + s0, S, m, delta, kv, yf, yr, rp);
      double* gl = gvec + (int64_t)l * S * g.nv;
#pragma unroll
      for (int k = 0; k < kSG; ++k) {
        if (s0 + k < S) {
          atomicAdd(gl + (s0 + k) * g.nv + bv, (double)(yf[k] * rp));
          atomicAdd(gl + (s0 + k) * g.nv + a, (double)(yr[k] * rp));
        }
      }
    }
  }
}

// U_v = sum_l w_l u_v^(l) in FP64; also leaves xw[l][v][s] = w_l u_v^(l) in the
// sweep precision for the interior recovery (sample-minor: an edge end's
// samples are one contiguous row).
// One CTA per tile of 32 vertices and 32 samples: for each node l the tile's
// FP64 solutions are read along the vertices ([l][s][v] rows) and the weighted
// values written along the samples ([l][v][s] rows) through a shared-memory
// transpose, so both sides stay coalesced; the FP64 node sum of every (s, v)
// stays in the registers of its thread. kAccL nodes are loaded before each
// transpose, so every thread has kAccL x 4 independent loads in flight.
constexpr int kAccTile = 32, kAccRows = 8, kAccS = 32, kAccL = 4;

template <typename T, typename OutT>
__global__ void __launch_bounds__(kAccTile * kAccRows)
    vertex_accum_kernel(DevGraph g, DevNodes nd, int64_t S, const double* __restrict__ xv,
                        OutT* __restrict__ out, T* __restrict__ xw) {
  __shared__ T tile[kAccL][kAccS][kAccTile + 1];
  const int tx = threadIdx.x % kAccTile, ty = threadIdx.x / kAccTile;
  const int64_t n_vt = (g.nv + kAccTile - 1) / kAccTile;
  const int64_t n_sc = (S + kAccS - 1) / kAccS;
  constexpr int kQ = kAccS / kAccRows;
  for (int64_t b = blockIdx.x; b < n_vt * n_sc; b += gridDim.x) {
    const int64_t v0 = (b % n_vt) * kAccTile, s0 = (b / n_vt) * kAccS;
    const int vn = (int)(g.nv - v0 < kAccTile ? g.nv - v0 : kAccTile);
    const int sn = (int)(S - s0 < kAccS ? S - s0 : kAccS);
    double acc[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) acc[q] = 0.0;
    for (int32_t l0 = 0; l0 < nd.L; l0 += kAccL) {
      const int nl = nd.L - l0 < kAccL ? nd.L - l0 : kAccL;
      double x[kAccL][kQ];
#pragma unroll
      for (int u = 0; u < kAccL; ++u)
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          const int s = ty + q * kAccRows;
          x[u][q] = (u < nl && s < sn && tx < vn)
                        ? xv[((int64_t)(l0 + u) * S + s0 + s) * g.nv + v0 + tx]
                        : 0.0;
        }
#pragma unroll
      for (int u = 0; u < kAccL; ++u) {
        const double wl = u < nl ? nd.weight[l0 + u] : 0.0;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          const double wx = wl * x[u][q];
          acc[q] += wx;
          tile[u][ty + q * kAccRows][tx] = (T)wx;
        }
      }
      __syncthreads();
      // the tile's rows xw[l][v0 + j][s0 .. s0 + sn) follow each other when
      // sn == S; write them along the samples
      for (int idx = threadIdx.x; idx < nl * vn * sn; idx += blockDim.x) {
        const int u = idx / (vn * sn), r = idx - u * vn * sn;
        const int j = r / sn, s = r - j * sn;
        xw[((int64_t)(l0 + u) * g.nv + v0 + j) * S + s0 + s] = tile[u][s][j];
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int s = ty + q * kAccRows;
      if (s < sn && tx < vn) out[(s0 + s) * g.n + v0 + tx] = (OutT)acc[q];
    }
  }
}

// The vertex values from weighted values the batched PCG wrote already
// (xw[l][v][s] = w_l u_v^(l), FP32): out(s, v) = sum over l, accumulated as an
// FP32 pair per value (about 48 bits, no FP64 instruction). One CTA per tile of
// 32 vertices x 32 samples: the lanes read along the samples, four rows of
// vertices per thread, and a transpose in shared memory writes along the
// vertices.
__device__ __forceinline__ void pair_add(float& h, float& l, float t) {
  const float s = __fadd_rn(h, t);
  const float bv = __fsub_rn(s, h);
  l = __fadd_rn(l, __fadd_rn(__fsub_rn(h, __fsub_rn(s, bv)), __fsub_rn(t, bv)));
  h = s;
}

template <typename OutT>
__global__ void __launch_bounds__(kAccTile * kAccRows)
    vertex_sum_kernel(DevGraph g, int32_t L, int64_t S, const float* __restrict__ xw,
                      OutT* __restrict__ out) {
  __shared__ float tile[kAccS][kAccTile + 1];
  const int tx = threadIdx.x % kAccTile, ty = threadIdx.x / kAccTile;
  const int64_t n_vt = (g.nv + kAccTile - 1) / kAccTile;
  const int64_t n_sc = (S + kAccS - 1) / kAccS;
  constexpr int kQ = kAccTile / kAccRows;
  const int64_t lstride = (int64_t)g.nv * S;
  for (int64_t b = blockIdx.x; b < n_vt * n_sc; b += gridDim.x) {
    const int64_t v0 = (b % n_vt) * kAccTile, s0 = (b / n_vt) * kAccS;
    const int vn = (int)(g.nv - v0 < kAccTile ? g.nv - v0 : kAccTile);
    const int sn = (int)(S - s0 < kAccS ? S - s0 : kAccS);
    float h[kQ], lo[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) h[q] = lo[q] = 0.f;
    const float* p = xw + (v0 + ty) * S + s0 + tx;
    if (tx < sn) {
      int32_t l = 0;
      for (; l + 4 <= L; l += 4) {
        float x[4][kQ];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int q = 0; q < kQ; ++q)
            x[u][q] = ty + q * kAccRows < vn ? __ldg(p + (l + u) * lstride + q * kAccRows * S)
                                             : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int q = 0; q < kQ; ++q) pair_add(h[q], lo[q], x[u][q]);
      }
      for (; l < L; ++l)
#pragma unroll
        for (int q = 0; q < kQ; ++q)
          if (ty + q * kAccRows < vn) pair_add(h[q], lo[q], __ldg(p + l * lstride + q * kAccRows * S));
    }
    if (sizeof(OutT) == 8) {
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        const int j = ty + q * kAccRows;
        if (tx < sn && j < vn) out[(s0 + tx) * g.n + v0 + j] = (OutT)((double)h[q] + (double)lo[q]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < kQ; ++q) tile[tx][ty + q * kAccRows] = h[q] + lo[q];
      __syncthreads();
      // thread (tx, ty): vertex v0 + tx of samples ty, ty + 8, ...
#pragma unroll
      for (int q = 0; q < kAccS / kAccRows; ++q) {
        const int s = ty + q * kAccRows;
        if (s < sn && tx < vn) out[(s0 + s) * g.n + v0 + tx] = (OutT)tile[s][tx];
      }
      __syncthreads();
    }
  }
}

// thread -> (e, sample group); loops over all nodes l, keeping the FP64 sum
// of w_l x^(l) in acc. yscr / rpscr hold the forward sweep for the back sweep.
template <typename T, typename OutT>
__global__ void recover_kernel(DevGraph g, DevNodes nd, double kappa2, int64_t S,
                               const int32_t* __restrict__ edges, int32_t n_edges,
                               const T* __restrict__ b, const double* __restrict__ xv,
                               OutT* __restrict__ out, double* __restrict__ acc,
                               T* __restrict__ yscr, T* __restrict__ rpscr) {
  const int64_t nsg = (S + kSG - 1) / kSG;
  const int64_t total = (int64_t)n_edges * nsg;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sg = t % nsg;
    const int32_t e = edges[t / nsg];
    const int32_t m = g.nel[e] - 1;
    if (m <= 0) continue;
    const int64_t off = g.ioff[e];
    const int64_t s0 = sg * kSG;
    const T* bI = b + (g.nv + off) * S;
    double* aI = acc + off * S;
    T* yI = yscr + off * S;
    T* rI = rpscr + off * nsg + sg;
    const double h = g.he[e];
    const int32_t va = g.eu[e], vb = g.ev[e];
    for (int32_t l = 0; l < nd.L; ++l) {
      const double gam = nd.gamma[l];
      const double w = nd.weight[l];
      const T delta = (T)((nd.alpha[l] / gam + kappa2) * h * h);
      const T sc = (T)(w * h / gam);  // w_l / c
      T xa[kSG], xb[kSG], y[kSG];
#pragma unroll
      for (int k = 0; k < kSG; ++k) {
        const bool ok = s0 + k < S;
        const int64_t base = ((int64_t)l * S + (ok ? s0 + k : 0)) * g.nv;
        xa[k] = ok ? (T)(w * xv[base + va]) : (T)0;
        xb[k] = ok ? (T)(w * xv[base + vb]) : (T)0;
        y[k] = ok ? bI[s0 + k] * sc + xa[k] + (m == 1 ? xb[k] : (T)0) : (T)0;
        if (ok) yI[s0 + k] = y[k];
      }
      T q = (T)1 + delta;
      T rp = (T)1 / ((T)1 + q);
      rI[0] = rp;
      for (int32_t i = 1; i < m; ++i) {
        const T* row = bI + (int64_t)i * S + s0;
        T* yrow = yI + (int64_t)i * S + s0;
        const bool last = (i == m - 1);
#pragma unroll
        for (int k = 0; k < kSG; ++k) {
          if (s0 + k < S) {
            y[k] = row[k] * sc + (last ? xb[k] : (T)0) + rp * y[k];
            yrow[k] = y[k];
          }
        }
        q = delta + q * rp;
        rp = (T)1 / ((T)1 + q);
        rI[(int64_t)i * nsg] = rp;
      }
      // back substitution, accumulating w_l x^(l) in FP64
      T x[kSG];
#pragma unroll
      for (int k = 0; k < kSG; ++k) {
        if (s0 + k < S) {
          x[k] = y[k] * rp;
          aI[(int64_t)(m - 1) * S + s0 + k] += (double)x[k];
        }
      }
      for (int32_t i = m - 2; i >= 0; --i) {
        const T rpi = rI[(int64_t)i * nsg];
        const T* yrow = yI + (int64_t)i * S + s0;
        double* arow = aI + (int64_t)i * S + s0;
#pragma unroll
        for (int k = 0; k < kSG; ++k) {
          if (s0 + k < S) {
            x[k] = (yrow[k] + x[k]) * rpi;
            arow[k] += (double)x[k];
          }
        }
      }
    }
    for (int32_t i = 0; i < m; ++i) {
#pragma unroll
      for (int k = 0; k < kSG; ++k) {
        if (s0 + k < S) out[(s0 + k) * g.n + g.nv + off + i] = (OutT)aI[(int64_t)i * S + s0 + k];
      }
    }
  }
}

template <typename T>
__global__ void to_minor_kernel(DevGraph g, int64_t S, const double* __restrict__ src,
                                T* __restrict__ dst, int mass_scale) {
  const int64_t total = S * g.n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / S;
    const int64_t s = t - j * S;
    double v = src[s * g.n + j];
    if (mass_scale) {
      const double r = g.sqrt_ml[j];
      v *= r * r;
    }
    dst[t] = (T)v;
  }
}

}  // namespace

int recover_sample_group() { return kSG; }

template <typename T>
int launch_condense(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S, const T* b,
                    double* gvec, cudaStream_t st, const int32_t* edges, int32_t n_edges,
                    bool init) {
  if (init)
    gvec_init_kernel<T><<<grid_for((int64_t)nd.L * S * g.nv, 256), 256, 0, st>>>(g, nd.L, S, b,
                                                                                 gvec);
  if (!edges) n_edges = g.ne;
  if (g.ni == 0 || n_edges == 0) return init ? 1 : 0;
  const int64_t nsg = (S + kSG - 1) / kSG;
  // one thread per node (rounded up to whole warps, at most 256 per pass)
  int threads = ((nd.L + 31) / 32) * 32;
  if (threads > 256) threads = 256;
  // stage edges up to 64 KB of rows (4096 FP32 rows of 4 samples); longer ones
  // stream from global memory
  const int32_t cap = (int32_t)((64 * 1024) / (kSG * sizeof(T)));
  const int32_t stage_max = g.max_m < cap ? g.max_m : cap;
  const size_t smem = (size_t)(stage_max > 0 ? stage_max : 1) * kSG * sizeof(T);
  cudaFuncSetAttribute(condense_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int64_t blocks = (int64_t)n_edges * nsg;
  if (blocks > sm_count() * 64) blocks = sm_count() * 64;
  condense_kernel<T><<<(int)blocks, threads, smem, st>>>(g, nd, kappa2, S, b, gvec, stage_max,
                                                         edges, n_edges);
  return init ? 2 : 1;
}

template <typename T, typename OutT>
int launch_recover(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S, const T* b,
                   const double* xv, OutT* out, const SweepParams<T>* prm, T* xw,
                   const int32_t* bin_edges, const int32_t* bin_count, int32_t n_bins, double* acc,
                   T* yscr, T* rpscr, int sg, cudaStream_t st, bool xw_ready) {
  {
    const int64_t tiles = ((g.nv + kAccTile - 1) / kAccTile) * ((S + kAccS - 1) / kAccS);
    if (xw_ready && sizeof(T) == 4)
      vertex_sum_kernel<OutT><<<grid_for(tiles * 256, 256), kAccTile * kAccRows, 0, st>>>(
          g, nd.L, S, (const float*)xw, out);
    else
      vertex_accum_kernel<T, OutT><<<grid_for(tiles * 256, 256), kAccTile * kAccRows, 0, st>>>(
          g, nd, S, xv, out, xw);
  }
  int launches = 1;
  if (g.ni == 0) return launches;
  launches +=
      launch_recover_bins<T, OutT>(g, nd.L, S, b, prm, xw, out, bin_edges, bin_count, sg, st);
  int64_t skip = 0;
  for (int i = 0; i < n_bins; ++i) skip += bin_count[i];
  const int32_t n_long = bin_count[n_bins];  // edges longer than the largest bin
  if (n_long > 0) {
    cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)g.ni * (size_t)S, st);
    const int64_t nsg = (S + kSG - 1) / kSG;
    recover_kernel<T, OutT><<<grid_for((int64_t)n_long * nsg, 128), 128, 0, st>>>(
        g, nd, kappa2, S, bin_edges + skip, n_long, b, xv, out, acc, yscr, rpscr);
    launches += 1;
  }
  return launches;
}

template <typename T>
void launch_to_minor(const DevGraph& g, int64_t S, const double* src, T* dst, bool mass_scale,
                     cudaStream_t st) {
  to_minor_kernel<T><<<grid_for(S * g.n, 256), 256, 0, st>>>(g, S, src, dst, mass_scale ? 1 : 0);
}

template int launch_condense<float>(const DevGraph&, const DevNodes&, double, int64_t,
                                    const float*, double*, cudaStream_t, const int32_t*,
                                    int32_t, bool);
template int launch_condense<double>(const DevGraph&, const DevNodes&, double, int64_t,
                                     const double*, double*, cudaStream_t, const int32_t*,
                                     int32_t, bool);
#define GRF_INST_RECOVER(T, O)                                                                 \
  template int launch_recover<T, O>(const DevGraph&, const DevNodes&, double, int64_t, const T*, \
                                    const double*, O*, const SweepParams<T>*, T*,                \
                                    const int32_t*, const int32_t*, int32_t, double*, T*, T*,    \
                                    int, cudaStream_t, bool);
GRF_INST_RECOVER(float, float)
GRF_INST_RECOVER(float, double)
GRF_INST_RECOVER(double, double)
GRF_INST_RECOVER(double, float)
#undef GRF_INST_RECOVER
template void launch_to_minor<float>(const DevGraph&, int64_t, const double*, float*, bool,
                                     cudaStream_t);
template void launch_to_minor<double>(const DevGraph&, int64_t, const double*, double*, bool,
                                      cudaStream_t);

}  // namespace grf
