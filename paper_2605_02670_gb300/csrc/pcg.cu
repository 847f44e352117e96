// Jacobi-preconditioned CG on the vertex Schur systems S^(l) u = g (Eq.
// global_schur; Sec. 3, Phase 4), one system per (node l, sample s).
//
// S^(l) is applied from its per-edge 2x2 blocks: y_v = D_v x_v + sum over the
// incidences k of v of offv_k x_{nbr(k)} (Eq. goal_func_1 with the blocks of
// Eq. local_reduced_schur). Stop when ||r||_2 <= rtol ||g||_2 or after
// max_iter iterations (counted as unconverged); a zero right-hand side gives
// u = 0.
//
// FP64 mode (VT = double): plain PCG in FP64, z = r * (1 / D) with the stored
// inverse diagonal.
// Mixed mode (VT = float): FP32 inner CG inside FP64 iterative refinement.
// Each refinement step forms the true residual r = g - S x in FP64 with the
// FP64 blocks and solves S d = r in FP32 in its Jacobi-scaled form
//   (D^-1/2 S D^-1/2) e = D^-1/2 r / sigma,   d = sigma D^-1/2 e,
// sigma = ||D^-1/2 r||, whose matrix has unit diagonal and off-diagonal
// entries offv_k / sqrt(D_v D_w) stored in FP32: every FP32 quantity is then
// O(1) whatever the shift (the raw entries span 1e-30 .. 1e+34 over the
// quadrature nodes). CG on the scaled matrix is Jacobi-PCG on S. The inner
// solve stops at a relative 1e-4 or when the FP32 recurrence stops improving;
// the stopping test is always on the FP64 residual, whose norms are FP64 dot
// products. The inner correction solve keeps its own dots and scalars (alpha,
// beta) in FP32. On GB300 FP64 arithmetic runs at a small fraction of the FP32
// rate, and even one thread's serial FP64 scalar work per iteration stalls
// the whole CTA, which is what this split is for.
//
// One CTA owns a system for its whole solve: the reductions are CTA-local
// (warp shuffles + shared memory), so no CTA ever waits on another and every
// loop is bounded by max_iter. Two layouts:
//   pcg_kernel: one system after another per CTA, matrix read through L1/L2,
//     vectors in shared memory when they fit (else global scratch);
//   pcg_staged_kernel (mixed mode, small graphs): one CTA per (node, group of
//     samples) stages that node's FP32 matrix and the incidence lists in
//     shared memory once and solves its samples from shared memory only.
#include "grf_internal.h"

namespace grf {
namespace {

constexpr size_t kSmemMax = 220 * 1024;
constexpr double kInnerRtol = 1e-4;

// Verdicts of the inner loop.
constexpr int kDone = 1, kStop = 2, kBad = 3;

template <int kThreads, int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* sh) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();  // previous readers of sh are done
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) sh[warp * N + k] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    double a = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) a += sh[w * N + k];
    v[k] = a;
  }
}

// Shuffle-reduce N per-thread partials within each warp; lane 0 stores the
// warp's sums in shw[warp * N + k].
template <typename VT, int N>
__device__ __forceinline__ void warp_partials(VT (&v)[N], VT* shw) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) shw[(threadIdx.x >> 5) * N + k] = v[k];
  }
}

// Sum over the warps of component k, in VT (every thread, same order)
template <int kThreads, typename VT>
__device__ __forceinline__ VT sum_partials(const VT* shw, int k, int N) {
  VT a = (VT)0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) a += shw[w * N + k];
  return a;
}

// Per-system vectors: VT d (update), r, p, q; FP64 x (the iterate) when
// refining; y (learned preconditioner only) holds B^T r.
template <typename VT>
struct SysVecs {
  VT *d, *r, *p, *q;
  double* x;
  VT* y;
};

// One node's matrix as seen by the solver. vptr/nbr/Ot/Ds may point to shared
// or global memory; D/O (FP64, refinement residual) are global.
template <typename VT>
struct SysMatrix {
  const int32_t* vptr;
  const int32_t* nbr;
  const VT* Ot;      // FP64 mode: the blocks; mixed: the scaled FP32 blocks
  const VT* Ds;      // FP64 mode: 1 / D; mixed: 1 / sqrt(D)
  const double* D;   // FP64 diagonal
  const double* O;   // FP64 blocks
  // learned preconditioner of the scaled system (mixed mode), else null:
  // B = diag(es) + N, N_{v, nbr k} = nb[k]; rev = reverse incidence
  const float* es;
  const float* nb;
  const int32_t* rev;
};

// z = B (B^T r) for the learned preconditioner: y_w = es_w r_w +
// sum_k' nb_{rev k'} r_{nbr k'}; z_v = es_v y_v + sum_k nb_k y_{nbr k}. Writes z
// and returns this thread's share of r.z; ends with all threads past a barrier.
template <int kThreads, typename VT>
__device__ __forceinline__ VT learned_apply(int32_t nv, const SysMatrix<VT>& M, const VT* r,
                                            VT* y, VT* z) {
  for (int32_t w = threadIdx.x; w < nv; w += kThreads) {
    VT acc = (VT)M.es[w] * r[w];
    for (int32_t k = M.vptr[w]; k < M.vptr[w + 1]; ++k)
      acc += (VT)M.nb[M.rev[k]] * r[M.nbr[k]];
    y[w] = acc;
  }
  __syncthreads();
  VT rz = (VT)0;
  for (int32_t v = threadIdx.x; v < nv; v += kThreads) {
    VT acc = (VT)M.es[v] * y[v];
    for (int32_t k = M.vptr[v]; k < M.vptr[v + 1]; ++k) acc += (VT)M.nb[k] * y[M.nbr[k]];
    z[v] = acc;
    rz += r[v] * acc;
  }
  return rz;
}

template <int kThreads, typename VT>
struct Shared {
  double sh[(kThreads / 32) * 2];
  VT shw[(kThreads / 32)];
  VT shw2[(kThreads / 32) * 2];
};

struct SysResult {
  int32_t it;
  bool done, bad, fallback;
};

// FP64 residual r_i = g_i - (S x)_i
template <typename VT>
__device__ __forceinline__ double residual(const SysMatrix<VT>& M, const double* gs,
                                           const double* x, int32_t i) {
  double y = M.D[i] * x[i];
  for (int32_t k = M.vptr[i]; k < M.vptr[i + 1]; ++k) y += M.O[k] * x[M.nbr[k]];
  return gs[i] - y;
}

// Solves one system S u = g (all threads of the CTA); writes u to xo.
template <int kThreads, typename VT>
__device__ SysResult solve_system(int32_t nv, const SysMatrix<VT>& M, const double* __restrict__ gs,
                                  double* __restrict__ xo, SysVecs<VT> v, bool x_is_out,
                                  double rtol, int32_t max_iter, Shared<kThreads, VT>& S) {
  constexpr bool kRefine = sizeof(VT) == 4;
  // FP64 mode: one PCG run on d (= u, since it starts from 0).
  // Mixed mode: x (FP64) accumulates the scaled FP32 updates of each step.
  double gg[2] = {0.0, 0.0};
  for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
    const double gv = gs[i];
    gg[0] += gv * gv;
    if (kRefine) {
      const double sv = gv * (double)M.Ds[i];
      gg[1] += sv * sv;
      v.x[i] = 0.0;
    }
    v.d[i] = (VT)0;
  }
  block_sum<kThreads, 2>(gg, S.sh);
  const double tol2 = rtol * rtol * gg[0];
  int32_t it = 0;
  bool bad = !isfinite(gg[0]) || !isfinite(gg[1]);
  bool done = bad || !(gg[0] > 0.0);
  double sig2 = gg[1];  // ||D^-1/2 r||^2 of the current refinement step
  // z = B B^T r (learned), else z = r on the scaled system (Jacobi). A learned
  // preconditioner that breaks down (r.z <= 0, p.Sp <= 0 or a non-finite
  // scalar) is dropped for the rest of this system's solve, which continues
  // with Jacobi from the last refined iterate.
  bool learned = kRefine && M.es != nullptr;
  bool fallback = false;
  while (!done && it < max_iter) {
    double sigma = 1.0;
    if (kRefine) {
      if (it > 0) {  // FP64 residual of the current iterate and its scaled norm
        __syncthreads();
        double acc[2] = {0.0, 0.0};
        for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
          const double ri = residual(M, gs, v.x, i);
          const double si = ri * (double)M.Ds[i];
          acc[0] += ri * ri;
          acc[1] += si * si;
        }
        block_sum<kThreads, 2>(acc, S.sh);
        if (!isfinite(acc[0]) || !isfinite(acc[1])) {
          bad = true;
          break;
        }
        if (acc[0] <= tol2) {
          done = true;
          break;
        }
        sig2 = acc[1];
      }
      if (!(sig2 > 0.0)) {
        done = true;
        break;
      }
      sigma = sqrt(sig2);
      const double inv = 1.0 / sigma;
      for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
        const double ri = it > 0 ? residual(M, gs, v.x, i) : gs[i];
        v.r[i] = (VT)(ri * (double)M.Ds[i] * inv);
        v.d[i] = (VT)0;
      }
      __syncthreads();
    } else {
      for (int32_t i = threadIdx.x; i < nv; i += kThreads) v.r[i] = (VT)gs[i];
    }
    // (P)CG on the inner system from d = 0
    VT rz0 = (VT)0;
    if (learned) {
      rz0 = learned_apply<kThreads, VT>(nv, M, v.r, v.y, v.p);
    } else {
      for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
        const VT ri = v.r[i];
        const VT z = kRefine ? ri : ri * M.Ds[i];
        v.p[i] = z;
        rz0 += ri * z;
      }
    }
    double a0[1] = {(double)rz0};
    block_sum<kThreads, 1>(a0, S.sh);
    // The CG scalars live in VT and every thread computes them from the same
    // per-warp partial sums in the same order, so all threads take the same
    // decisions without a broadcast (FP64 mode: FP64 dots; mixed mode: the
    // inner correction solve's dots in FP32, the outer residual norms above in
    // FP64). Two partial-sum buffers alternate so that three barriers per
    // iteration suffice.
    VT rz = (VT)a0[0];
    // inner stop: mixed relative to the unit start, FP64 on the true residual
    const VT inner2 = kRefine ? (VT)(kInnerRtol * kInnerRtol) : (VT)tol2;
    VT best = kRefine ? (VT)1 : (VT)gg[0];
    int since_best = 0;
    int verdict = learned && !(rz > (VT)0 && isfinite((double)rz)) ? kBad : 0;
    while (verdict == 0 && it < max_iter) {
      ++it;
      __syncthreads();  // p from the previous update is visible
      VT pqf = (VT)0;
      for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
        VT y = kRefine ? v.p[i] : (VT)M.D[i] * v.p[i];
        for (int32_t k = M.vptr[i]; k < M.vptr[i + 1]; ++k) y += M.Ot[k] * v.p[M.nbr[k]];
        v.q[i] = y;
        pqf += v.p[i] * y;
      }
      VT part1[1] = {pqf};
      warp_partials<VT, 1>(part1, S.shw);
      __syncthreads();
      const VT pq = sum_partials<kThreads, VT>(S.shw, 0, 1);
      if (!isfinite((double)pq)) {
        verdict = kBad;
        break;
      }
      if (!(pq > (VT)0)) {  // p vanished (mixed: at the FP32 floor)
        verdict = kRefine && !learned ? kStop : kBad;
        break;
      }
      const VT af = rz / pq;
      VT rzf = (VT)0, rrf = (VT)0;
      for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
        v.d[i] += af * v.p[i];
        const VT ri = v.r[i] - af * v.q[i];
        v.r[i] = ri;
        rzf += kRefine ? ri * ri : ri * ri * M.Ds[i];
        rrf += ri * ri;
      }
      if (learned) {  // z = B B^T r into q (q is consumed above)
        __syncthreads();
        rzf = learned_apply<kThreads, VT>(nv, M, v.r, v.y, v.q);
      }
      VT part2[2] = {rzf, rrf};
      warp_partials<VT, 2>(part2, S.shw2);
      __syncthreads();
      const VT rzn = sum_partials<kThreads, VT>(S.shw2, 0, 2);
      const VT rr = sum_partials<kThreads, VT>(S.shw2, 1, 2);
      if (!isfinite((double)rzn) || !isfinite((double)rr)) {
        verdict = kBad;
        break;
      }
      if (rr <= inner2) {
        verdict = kDone;
        break;
      }
      if (kRefine) {  // the FP32 recurrence has reached its rounding floor
        if (rr < (VT)0.98 * best) {
          best = rr;
          since_best = 0;
        } else if (++since_best >= 32) {
          verdict = kStop;
          break;
        }
      }
      const VT bf = rzn / rz;
      rz = rzn;
      for (int32_t i = threadIdx.x; i < nv; i += kThreads)
        v.p[i] = (learned ? v.q[i] : (kRefine ? v.r[i] : v.r[i] * M.Ds[i])) + bf * v.p[i];
    }
    const bool inner_done = verdict == kDone;
    if (verdict == kBad && learned) {  // drop the correction, go on with Jacobi
      learned = false;
      fallback = true;
      continue;
    }
    if (verdict == kBad) bad = true;
    if (bad) break;
    if (!kRefine) {
      done = inner_done;
      break;
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i < nv; i += kThreads)
      v.x[i] += sigma * (double)M.Ds[i] * (double)v.d[i];
  }
  if (kRefine && !done && !bad) {
    // iteration budget spent: test the FP64 residual of the final iterate
    __syncthreads();
    double acc[1] = {0.0};
    for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
      const double ri = residual(M, gs, v.x, i);
      acc[0] += ri * ri;
    }
    block_sum<kThreads, 1>(acc, S.sh);
    done = acc[0] <= tol2;
  }
  __syncthreads();
  if (kRefine) {
    if (!x_is_out)
      for (int32_t i = threadIdx.x; i < nv; i += kThreads) xo[i] = v.x[i];
  } else {
    for (int32_t i = threadIdx.x; i < nv; i += kThreads) xo[i] = (double)v.d[i];
  }
  return SysResult{it, done, bad, fallback};
}

template <int kThreads>
__device__ __forceinline__ void report(int64_t sys, const SysResult& r, int32_t* iters,
                                       PcgStatus* status) {
  if (threadIdx.x == 0) {
    iters[sys] = r.it;
    atomicAdd(&status->iters_total, (unsigned long long)r.it);
    atomicMax(&status->iters_max, r.it);
    if (r.fallback) atomicAdd(&status->n_fallback, 1);
    if (r.bad) atomicAdd(&status->numeric_flag, 1);
    else if (!r.done) atomicAdd(&status->n_unconverged, 1);
  }
}

constexpr int kThreadsA = 256;

// dscale: FP64 mode 1 / D; mixed mode 1 / sqrt(D).
// offv_t: FP64 mode the blocks; mixed mode the Jacobi-scaled blocks.
// lp_es / lp_n (mixed mode, may be null): learned preconditioner per node,
// diag(es) [L][V] and the incidence entries [L][2E].
template <typename VT, bool kSmem>
__global__ void __launch_bounds__(kThreadsA) pcg_kernel(
    DevGraph g, int32_t L, int64_t S, const double* __restrict__ diag,
    const double* __restrict__ offv, const VT* __restrict__ dscale_t,
    const VT* __restrict__ offv_t, const float* __restrict__ lp_es,
    const float* __restrict__ lp_n, const double* __restrict__ gvec, double* __restrict__ xout,
    VT* __restrict__ gd, VT* __restrict__ gr, VT* __restrict__ gp, VT* __restrict__ gq,
    VT* __restrict__ gy, double rtol, int32_t max_iter, int32_t* __restrict__ iters,
    PcgStatus* status) {
  constexpr bool kRefine = sizeof(VT) == 4;
  __shared__ Shared<kThreadsA, VT> shs;
  extern __shared__ __align__(16) unsigned char vec_sm[];
  const int64_t nsys = (int64_t)L * S;
  const int32_t nv = g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  for (int64_t sys = blockIdx.x; sys < nsys; sys += gridDim.x) {
    const int64_t l = sys / S;
    SysMatrix<VT> M{g.vptr,
                    g.adj_nbr,
                    offv_t + l * ne2,
                    dscale_t + l * nv,
                    diag + l * nv,
                    offv + l * ne2,
                    lp_es ? lp_es + l * nv : nullptr,
                    lp_n ? lp_n + l * ne2 : nullptr,
                    g.adj_rev};
    double* xo = xout + sys * nv;
    SysVecs<VT> v;
    if (kSmem) {
      v.x = reinterpret_cast<double*>(vec_sm);
      VT* base = reinterpret_cast<VT*>(vec_sm + (kRefine ? sizeof(double) * nv : 0));
      v.d = base;
      v.r = base + nv;
      v.p = base + 2 * (int64_t)nv;
      v.q = base + 3 * (int64_t)nv;
      v.y = base + 4 * (int64_t)nv;  // allocated only with the learned preconditioner
    } else {
      v.x = xo;
      v.d = gd + sys * nv;
      v.r = gr + sys * nv;
      v.p = gp + sys * nv;
      v.q = gq + sys * nv;
      v.y = gy + sys * nv;
    }
    const SysResult res = solve_system<kThreadsA, VT>(nv, M, gvec + sys * nv, xo, v, !kSmem,
                                                      rtol, max_iter, shs);
    report<kThreadsA>(sys, res, iters, status);
    __syncthreads();
  }
}

constexpr int kThreadsB = 512;

// Shared memory of the staged kernel: matrix (vptr, nbr, scaled FP32 blocks,
// 1 / sqrt(D)) then the vectors (FP64 x; FP32 d, r, p, q).
__host__ __device__ inline size_t staged_bytes(int32_t nv, int32_t ne) {
  const size_t a = 4 * ((size_t)nv + 1) + 4 * 2 * (size_t)ne + 4 * 2 * (size_t)ne + 4 * (size_t)nv;
  const size_t a16 = (a + 15) & ~(size_t)15;
  return a16 + 8 * (size_t)nv + 4 * 4 * (size_t)nv;
}

__global__ void __launch_bounds__(kThreadsB) pcg_staged_kernel(
    DevGraph g, int32_t L, int64_t S, int32_t chunk, const double* __restrict__ diag,
    const double* __restrict__ offv, const float* __restrict__ dscale_t,
    const float* __restrict__ offv_t, const double* __restrict__ gvec, double* __restrict__ xout,
    double rtol, int32_t max_iter, int32_t* __restrict__ iters, PcgStatus* status) {
  __shared__ Shared<kThreadsB, float> shs;
  extern __shared__ __align__(16) unsigned char sm[];
  const int32_t nv = g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  int32_t* vptr = reinterpret_cast<int32_t*>(sm);
  int32_t* nbr = vptr + nv + 1;
  float* Ot = reinterpret_cast<float*>(nbr + ne2);
  float* Ds = Ot + ne2;
  const size_t a = 4 * ((size_t)nv + 1) + 8 * (size_t)ne2 + 4 * (size_t)nv;
  unsigned char* vb = sm + ((a + 15) & ~(size_t)15);
  SysVecs<float> v;
  v.x = reinterpret_cast<double*>(vb);
  v.d = reinterpret_cast<float*>(v.x + nv);
  v.r = v.d + nv;
  v.p = v.r + nv;
  v.q = v.p + nv;
  v.y = nullptr;
  const int64_t nchunk = (S + chunk - 1) / chunk;
  const int64_t units = (int64_t)L * nchunk;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t l = u / nchunk;
    const int64_t s_begin = (u % nchunk) * chunk;
    const int64_t s_end = s_begin + chunk < S ? s_begin + chunk : S;
    __syncthreads();  // the previous unit is done with the staged matrix
    for (int32_t i = threadIdx.x; i <= nv; i += kThreadsB) vptr[i] = g.vptr[i];
    for (int64_t k = threadIdx.x; k < ne2; k += kThreadsB) {
      nbr[k] = g.adj_nbr[k];
      Ot[k] = offv_t[l * ne2 + k];
    }
    for (int32_t i = threadIdx.x; i < nv; i += kThreadsB) Ds[i] = dscale_t[l * nv + i];
    __syncthreads();
    SysMatrix<float> M{vptr, nbr, Ot, Ds, diag + l * nv, offv + l * ne2, nullptr, nullptr,
                       nullptr};
    for (int64_t s = s_begin; s < s_end; ++s) {
      const int64_t sys = l * S + s;
      const SysResult res = solve_system<kThreadsB, float>(nv, M, gvec + sys * nv,
                                                           xout + sys * nv, v, false, rtol,
                                                           max_iter, shs);
      report<kThreadsB>(sys, res, iters, status);
      __syncthreads();
    }
  }
}

}  // namespace

template <typename VT>
void launch_pcg(const DevGraph& g, int32_t L, int64_t S, const double* diag, const double* offv,
                const VT* dscale_t, const VT* offv_t, const float* lp_es, const float* lp_n,
                const double* gvec, double* x, VT* d, VT* r, VT* p, VT* q, VT* y, double rtol,
                int32_t max_iter, int32_t* iters, PcgStatus* status, int layout,
                cudaStream_t st) {
  const int64_t nsys = (int64_t)L * S;
  if constexpr (sizeof(VT) == 4) {
    const size_t sb = staged_bytes(g.nv, g.ne) + sizeof(Shared<kThreadsB, float>);
    if (sb <= kSmemMax && layout == 2 && !lp_es) {
      // enough (node, sample-group) units to fill the GPU, one CTA per SM
      int64_t groups = (2 * 152 + L - 1) / L;
      if (groups > S) groups = S;
      if (groups < 1) groups = 1;
      const int32_t chunk = (int32_t)((S + groups - 1) / groups);
      const int64_t units = (int64_t)L * ((S + chunk - 1) / chunk);
      const size_t dyn = staged_bytes(g.nv, g.ne);
      cudaFuncSetAttribute(pcg_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)dyn);
      const int blocks = (int)(units < 152 * 8 ? units : 152 * 8);
      pcg_staged_kernel<<<blocks, kThreadsB, dyn, st>>>(g, L, S, chunk, diag, offv, dscale_t,
                                                        offv_t, gvec, x, rtol, max_iter, iters,
                                                        status);
      return;
    }
  }
  int blocks = (int)(nsys < 152 * 16 ? nsys : 152 * 16);
  if (blocks < 1) blocks = 1;
  const size_t smem = (sizeof(VT) == 4 ? sizeof(double) : 0) * (size_t)g.nv +
                      (lp_es ? 5 : 4) * sizeof(VT) * (size_t)g.nv;
  if (smem <= kSmemMax - 16 * 1024) {
    // dynamic + static may pass the 48 KB default; per device: set at every launch
    cudaFuncSetAttribute(pcg_kernel<VT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    pcg_kernel<VT, true><<<blocks, kThreadsA, smem, st>>>(g, L, S, diag, offv, dscale_t, offv_t,
                                                          lp_es, lp_n, gvec, x, d, r, p, q, y,
                                                          rtol, max_iter, iters, status);
  } else {
    pcg_kernel<VT, false><<<blocks, kThreadsA, 0, st>>>(g, L, S, diag, offv, dscale_t, offv_t,
                                                        lp_es, lp_n, gvec, x, d, r, p, q, y,
                                                        rtol, max_iter, iters, status);
  }
}
#define GRF_INST(VT)                                                                          \
  template void launch_pcg<VT>(const DevGraph&, int32_t, int64_t, const double*, const double*, \
                               const VT*, const VT*, const float*, const float*, const double*,  \
                               double*, VT*, VT*, VT*, VT*, VT*, double, int32_t, int32_t*,      \
                               PcgStatus*, int, cudaStream_t);
GRF_INST(float)
GRF_INST(double)
#undef GRF_INST

}  // namespace grf
