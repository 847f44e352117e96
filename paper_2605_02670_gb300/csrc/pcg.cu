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
// solve stops at a relative 1e-5 (or a tenth of the reduction still needed) or
// when the FP32 recurrence stops improving;
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
//   pcg_group_kernel (mixed mode, graphs up to 4096 vertices): one CTA per
//     (node, group of 2 or 4 samples) stages that node's FP32 matrix in shared
//     memory and runs the group's samples together, so every matrix load
//     serves the whole group; per-vertex vectors live in registers of the
//     owning thread, only the search directions are shared.
#include "grf_internal.h"

namespace grf {
namespace {

constexpr size_t kSmemMax = 220 * 1024;
constexpr double kInnerRtol = 1e-5;

// Verdicts of the inner loop.
constexpr int kDone = 1, kStop = 2, kBad = 3;

// Block sums of N doubles (sh: ((kThreads / 32) + 1) * N doubles). Thread k < N
// adds the per-warp partials of value k (FP64 runs at a small fraction of the
// FP32 rate on GB300, so every thread summing every partial would cost far
// more than the extra barrier).
template <int kThreads, int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* sh) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  constexpr int W = kThreads / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();  // previous readers of sh are done
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) sh[warp * N + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < N) {
    double a = 0.0;
    for (int w = 0; w < W; ++w) a += sh[w * N + threadIdx.x];
    sh[W * N + threadIdx.x] = a;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = sh[W * N + k];
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
  // preconditioner: kPreJacobi, kPreNeumann (z_v = pc_v r_v + sum_k pn_k r_nbr(k))
  // or kPreLearned (z = B B^T r, B = diag(pc) + N, N_{v, nbr k} = pn[k]);
  // rev = reverse incidence
  int pre;
  const VT* pc;
  const VT* pn;
  const int32_t* rev;
};

// z = P r for the sparse preconditioners (r must be complete: call after a
// barrier). Neumann-Neumann: one sweep. Learned: y_w = pc_w r_w +
// sum_k' pn_{rev k'} r_{nbr k'}, barrier, z_v = pc_v y_v + sum_k pn_k y_{nbr k}.
// Writes z and returns this thread's share of r.z.
template <int kThreads, typename VT>
__device__ __forceinline__ VT prec_apply(int32_t nv, const SysMatrix<VT>& M, const VT* r, VT* y,
                                         VT* z) {
  const VT* src = r;
  if (M.pre == kPreLearned) {
    for (int32_t w = threadIdx.x; w < nv; w += kThreads) {
      VT acc = M.pc[w] * r[w];
      for (int32_t k = M.vptr[w]; k < M.vptr[w + 1]; ++k) acc += M.pn[M.rev[k]] * r[M.nbr[k]];
      y[w] = acc;
    }
    __syncthreads();
    src = y;
  }
  VT rz = (VT)0;
  for (int32_t v = threadIdx.x; v < nv; v += kThreads) {
    VT acc = M.pc[v] * src[v];
    for (int32_t k = M.vptr[v]; k < M.vptr[v + 1]; ++k) acc += M.pn[k] * src[M.nbr[k]];
    z[v] = acc;
    rz += r[v] * acc;
  }
  return rz;
}

template <int kThreads, typename VT>
struct Shared {
  double sh[(kThreads / 32 + 1) * 2];
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
  double inner_e = kInnerRtol;  // relative stop of the current inner solve
  // z = P r (Neumann-Neumann or learned), else Jacobi (z = r on the scaled
  // system, r / D in FP64). A preconditioner that breaks down (r.z <= 0,
  // p.Sp <= 0 or a non-finite scalar) is dropped for the rest of this
  // system's solve, which continues with Jacobi from the last refined iterate.
  bool learned = M.pre != kPreJacobi;
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
        // solve the correction only as far as this step needs (a tenth of the
        // remaining ratio), never tighter than the FP32 floor
        inner_e = fmax(kInnerRtol, 0.1 * sqrt(tol2 / acc[0]));
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
    } else {  // FP64: one PCG run from d = 0 (again from 0 after a fallback)
      for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
        v.r[i] = (VT)gs[i];
        v.d[i] = (VT)0;
      }
    }
    // (P)CG on the inner system from d = 0
    VT rz0 = (VT)0;
    if (learned) {
      __syncthreads();
      rz0 = prec_apply<kThreads, VT>(nv, M, v.r, v.y, v.p);
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
    const VT inner2 = kRefine ? (VT)(inner_e * inner_e) : (VT)tol2;
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
        rzf = prec_apply<kThreads, VT>(nv, M, v.r, v.y, v.q);
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
// per-system CTAs with the vectors in global memory (measured on GB300: 128 and
// 512 threads per system both slower than 256 on 20 000- and 90 000-vertex graphs)
constexpr int kThreadsL = 256;

// dscale: FP64 mode 1 / D; mixed mode 1 / sqrt(D).
// offv_t: FP64 mode the blocks; mixed mode the Jacobi-scaled blocks.
// pre / pc / pn: preconditioner kind and its per-node coefficients
// ([L][V] and [L][2E]; see launch_pcg).
template <typename VT, bool kSmem, int NT>
__global__ void __launch_bounds__(NT) pcg_kernel(
    DevGraph g, int32_t L, int64_t S, const double* __restrict__ diag,
    const double* __restrict__ offv, const VT* __restrict__ dscale_t,
    const VT* __restrict__ offv_t, int pre, const VT* __restrict__ pc,
    const VT* __restrict__ pn, const double* __restrict__ gvec, double* __restrict__ xout,
    VT* __restrict__ gd, VT* __restrict__ gr, VT* __restrict__ gp, VT* __restrict__ gq,
    VT* __restrict__ gy, double rtol, int32_t max_iter, int32_t* __restrict__ iters,
    PcgStatus* status) {
  constexpr bool kRefine = sizeof(VT) == 4;
  __shared__ Shared<NT, VT> shs;
  extern __shared__ __align__(16) unsigned char vec_sm[];
  const int64_t nsys = (int64_t)L * S;
  const int32_t nv = g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  for (int64_t sys_i = blockIdx.x; sys_i < nsys; sys_i += gridDim.x) {
    const int64_t sys = nsys - 1 - sys_i;  // largest shifts first (longest solves)
    const int64_t l = sys / S;
    SysMatrix<VT> M{g.vptr,
                    g.adj_nbr,
                    offv_t + l * ne2,
                    dscale_t + l * nv,
                    diag + l * nv,
                    offv + l * ne2,
                    pre,
                    pre != kPreJacobi ? pc + l * nv : nullptr,
                    pre != kPreJacobi ? pn + l * ne2 : nullptr,
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
    const SysResult res = solve_system<NT, VT>(nv, M, gvec + sys * nv, xo, v, !kSmem, rtol,
                                               max_iter, shs);
    report<NT>(sys, res, iters, status);
    __syncthreads();
  }
}

constexpr int kThreadsG = 512;

// Shared memory of the group kernel: P [nv][SGP] (search directions of the
// group's samples, interleaved), the node's incidences as (neighbour, scaled
// FP32 off-diagonal) pairs [2E], 1 / sqrt(D) [nv] and the incidence offsets.
template <int SGP>
__host__ __device__ inline size_t group_bytes(int32_t nv, int32_t ne) {
  return 8 * (size_t)nv * SGP +
         4 * ((size_t)nv * SGP + 4 * (size_t)ne + (size_t)nv + (size_t)nv + 1) + 16;
}


// One vertex's row of the interleaved search directions (SGP floats, 8- or
// 16-byte aligned): a single vector access per vertex, no bank conflicts
// from strided scalar accesses.
template <int SGP>
__device__ __forceinline__ void load_row(const float* p, float (&v)[SGP]) {
  if constexpr (SGP == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  }
}
template <int SGP>
__device__ __forceinline__ void store_row(float* p, const float (&v)[SGP]) {
  if constexpr (SGP == 4)
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
}

// z = P r for the owned vertices of the group kernels (R holds every
// vertex's r, complete behind a barrier that this function starts with).
// Neumann-Neumann: z_v = pc_v r_v + sum_k pn_k r_nbr(k). Learned: Y = B^T r
// (barrier), z = B Y. Samples whose preconditioner is off get z = r. Returns
// rz[s] = r.z and rz[SGP + s] = r.r (thread partials).
template <int NT, int VPT, int SGP, bool kLearned>
__device__ __forceinline__ void prec_group_apply(const DevGraph& g, int32_t nv,
                                                 const int32_t* vp, const float* Pc,
                                                 const float* Pn, const float* R, float* Y,
                                                 const float (&r)[VPT][SGP],
                                                 const bool (&on)[SGP], float (&z)[VPT][SGP],
                                                 float (&rz)[2 * SGP]) {
  __syncthreads();  // R complete
  const float* src = R;
  if constexpr (kLearned) {
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const int32_t w = threadIdx.x + k * NT;
      if (w < nv) {
        float acc[SGP], rw[SGP];
        load_row<SGP>(R + (size_t)w * SGP, rw);
        const float c = Pc[w];
#pragma unroll
        for (int s = 0; s < SGP; ++s) acc[s] = c * rw[s];
        for (int32_t kk = vp[w]; kk < vp[w + 1]; ++kk) {
          const float o = Pn[g.adj_rev[kk]];
          float rv[SGP];
          load_row<SGP>(R + (size_t)g.adj_nbr[kk] * SGP, rv);
#pragma unroll
          for (int s = 0; s < SGP; ++s) acc[s] = fmaf(o, rv[s], acc[s]);
        }
        store_row<SGP>(Y + (size_t)w * SGP, acc);
      }
    }
    __syncthreads();  // Y complete
    src = Y;
  }
#pragma unroll
  for (int s = 0; s < 2 * SGP; ++s) rz[s] = 0.f;
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    const int32_t v = threadIdx.x + k * NT;
    if (v < nv) {
      float acc[SGP], sv[SGP];
      load_row<SGP>(src + (size_t)v * SGP, sv);
      const float c = Pc[v];
#pragma unroll
      for (int s = 0; s < SGP; ++s) acc[s] = c * sv[s];
      for (int32_t kk = vp[v]; kk < vp[v + 1]; ++kk) {
        const float o = Pn[kk];
        float sw[SGP];
        load_row<SGP>(src + (size_t)g.adj_nbr[kk] * SGP, sw);
#pragma unroll
        for (int s = 0; s < SGP; ++s) acc[s] = fmaf(o, sw[s], acc[s]);
      }
#pragma unroll
      for (int s = 0; s < SGP; ++s) {
        const float zs = on[s] ? acc[s] : r[k][s];
        z[k][s] = zs;
        rz[s] = fmaf(r[k][s], zs, rz[s]);
        rz[SGP + s] = fmaf(r[k][s], r[k][s], rz[SGP + s]);
      }
    } else {
#pragma unroll
      for (int s = 0; s < SGP; ++s) z[k][s] = 0.f;
    }
  }
}

// A vertex's row of the shared FP64 iterates (SGP doubles, 16-byte aligned).
template <int SGP>
__device__ __forceinline__ void load_xrow(const double* p, double (&v)[SGP]) {
#pragma unroll
  for (int s = 0; s < SGP; s += 2) {
    const double2 t = *reinterpret_cast<const double2*>(p + s);
    v[s] = t.x;
    v[s + 1] = t.y;
  }
}

// FP64 residual res[s] = g_s - (S x_s)_v of an owned vertex for the group's
// samples, from the shared FP64 iterates X [nv][SGP] and the node's FP64 blocks.
// The shared arrays are in slot order (slot v holds vertex ov), the global ones
// in vertex order: the incidences of slot v are vp[v] .. vp[v + 1] in NO and
// obeg onwards in O. Every incidence's coefficient and neighbour are loaded
// once for all samples, two incidences per step so that their loads are in
// flight together.
template <int SGP>
__device__ __forceinline__ void group_residual(int32_t v, int32_t ov, int32_t obeg, int32_t nv,
                                               const int32_t* vp, const int2* NO, const double* D,
                                               const double* O, const double* X, const double* gl,
                                               const bool (&act)[SGP], double (&res)[SGP]) {
  double y[SGP], xv[SGP];
  load_xrow<SGP>(X + (size_t)v * SGP, xv);
  const double dv = D[ov];
#pragma unroll
  for (int s = 0; s < SGP; ++s) y[s] = dv * xv[s];
  const int32_t kbeg = vp[v], kend = vp[v + 1];
  const double* Ov = O + obeg;
  int32_t kk = kbeg;
  for (; kk + 1 < kend; kk += 2) {
    const int32_t w0 = NO[kk].x, w1 = NO[kk + 1].x;
    const double o0 = Ov[kk - kbeg], o1 = Ov[kk + 1 - kbeg];
    double x0[SGP], x1[SGP];
    load_xrow<SGP>(X + (size_t)w0 * SGP, x0);
    load_xrow<SGP>(X + (size_t)w1 * SGP, x1);
#pragma unroll
    for (int s = 0; s < SGP; ++s)
      if (act[s]) y[s] = fma(o1, x1[s], fma(o0, x0[s], y[s]));
  }
  if (kk < kend) {
    const int32_t w0 = NO[kk].x;
    const double o0 = Ov[kk - kbeg];
    double x0[SGP];
    load_xrow<SGP>(X + (size_t)w0 * SGP, x0);
#pragma unroll
    for (int s = 0; s < SGP; ++s)
      if (act[s]) y[s] = fma(o0, x0[s], y[s]);
  }
#pragma unroll
  for (int s = 0; s < SGP; ++s) res[s] = act[s] ? gl[(int64_t)s * nv + ov] - y[s] : 0.0;
}

// Block sums of N floats (N = 2, 4 or 8) for NT <= 1024 threads: a warp
// butterfly, one row of N partials per warp in shared memory (16-byte aligned
// rows), then every warp reads the rows back with lane i taking row i mod W
// and finishes with a butterfly over W lanes (W = NT / 32). All warps run the
// same operations on the same data, so every thread ends with identical sums.
template <int NT, int N>
__device__ __forceinline__ void group_sum(float (&v)[N], float* shw) {
  constexpr int W = NT / 32;
#pragma unroll
  for (int k = 0; k < N; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < N; k += 2)
      *reinterpret_cast<float2*>(shw + (threadIdx.x >> 5) * N + k) = make_float2(v[k], v[k + 1]);
  }
  __syncthreads();
  const int row = (threadIdx.x & 31) % W;
#pragma unroll
  for (int k = 0; k < N; k += 2) {
    const float2 t = *reinterpret_cast<const float2*>(shw + row * N + k);
    v[k] = t.x;
    v[k + 1] = t.y;
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
}

// Mixed-precision PCG for one node and a group of SGP samples at a time: the
// same FP32 Jacobi-scaled inner CG inside FP64 refinement as solve_system,
// run for the group's samples together so that every load of the node's
// matrix serves SGP samples. Thread t owns slots t + k * NT
// (k < VPT): their r, q and d stay in registers; only the search directions,
// which neighbours read, are shared. Each sample keeps its own scalars,
// stopping tests and iteration count; the CTA iterates while any sample of the
// group is still working (every loop bounded by max_iter). The shared arrays
// hold the vertices in reverse Cuthill-McKee order (slot i is vertex
// ord.perm[i]), so that the rows a warp gathers lie in a narrow band of P.
template <int NT, int VPT, int SGP>
__global__ void __launch_bounds__(NT) pcg_group_kernel(
    DevGraph g, VertexOrder ord, int32_t L, int64_t S, const double* __restrict__ diag,
    const double* __restrict__ offv, const float* __restrict__ dscale_t,
    const float* __restrict__ offv_t, const double* __restrict__ gvec, double* __restrict__ xout,
    double rtol, int32_t max_iter, int32_t* __restrict__ iters, PcgStatus* status) {
  static_assert(SGP == 2 || SGP == 4, "sample groups of 2 or 4");
  __shared__ __align__(16) float shw[2][(NT / 32) * 2 * SGP];
  __shared__ double shd[(NT / 32 + 1) * 2 * SGP];
  // Per-sample scalars, written by thread 0. The refinement residual r is
  // carried in FP32 in two normalised forms: r / ||g|| (stop test against
  // rtol) and D^-1/2 r / sigma0 (sigma0 = ||D^-1/2 g||), so only S x and g - S x
  // need FP64. igd = 1 / ||g||, cgs = ||g|| / sigma0, sgm = sigma of the
  // current step, isg = sigma0 / sigma, in2 = inner stop.
  __shared__ double igd[SGP], sgm0[SGP], isg0[SGP], sgm[SGP];
  __shared__ float cgs[SGP], isg[SGP], in2[SGP];
  extern __shared__ __align__(16) unsigned char grp_sm[];
  const int32_t nv = g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  double* X = reinterpret_cast<double*>(grp_sm);  // [nv][SGP] FP64 iterates
  float* P = reinterpret_cast<float*>(X + (size_t)nv * SGP);  // [nv][SGP]
  int2* NO = reinterpret_cast<int2*>(P + (size_t)nv * SGP);  // [2E] (neighbour, bits of o)
  float* Ds = reinterpret_cast<float*>(NO + ne2);  // [nv]
  int32_t* vp = reinterpret_cast<int32_t*>(Ds + nv);  // [nv + 1] incidence offsets
  for (int32_t v = threadIdx.x; v <= nv; v += NT) vp[v] = ord.vptr[v];
  const int64_t ngrp = (S + SGP - 1) / SGP;
  const int64_t units = (int64_t)L * ngrp;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    // nodes from the largest shift down: the nodes that need the most
    // iterations start first, so the last wave is made of short solves
    const int64_t l = L - 1 - u / ngrp;
    const int64_t s0 = (u % ngrp) * SGP;
    const int kv = (int)(S - s0 < SGP ? S - s0 : SGP);
    __syncthreads();  // the previous unit is done with the shared arrays
    for (int64_t k = threadIdx.x; k < ne2; k += NT)
      NO[k] = make_int2(ord.nbr[k], __float_as_int(offv_t[l * ne2 + ord.inc[k]]));
    for (int32_t v = threadIdx.x; v < nv; v += NT) Ds[v] = dscale_t[l * nv + ord.perm[v]];
    __syncthreads();
    const double* D = diag + l * nv;
    const double* O = offv + l * ne2;
    const double* gl = gvec + (l * S + s0) * nv;  // sample s at gl + s * nv
    double* xl = xout + (l * S + s0) * nv;
    double nrm[2 * SGP];
#pragma unroll
    for (int s = 0; s < 2 * SGP; ++s) nrm[s] = 0.0;
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const int32_t v = threadIdx.x + k * NT;
      if (v < nv) {
        const int32_t ov = ord.perm[v];
#pragma unroll
        for (int s = 0; s < SGP; ++s) {
          if (s < kv) {
            const double gv = gl[(int64_t)s * nv + ov];
            const double sv = gv * (double)Ds[v];
            nrm[s] += gv * gv;
            nrm[SGP + s] += sv * sv;
          }
          X[(size_t)v * SGP + s] = 0.0;
        }
      }
    }
    block_sum<NT, 2 * SGP>(nrm, shd);
    bool act[SGP], done[SGP], bad[SGP];
    int32_t its[SGP];
    if (threadIdx.x == 0) {
#pragma unroll
      for (int s = 0; s < SGP; ++s) {
        const double gn = sqrt(nrm[s]);
        sgm0[s] = sqrt(nrm[SGP + s]);
        isg0[s] = sgm0[s] > 0.0 ? 1.0 / sgm0[s] : 0.0;
        sgm[s] = sgm0[s];
        igd[s] = gn > 0.0 ? 1.0 / gn : 0.0;
        cgs[s] = sgm0[s] > 0.0 ? (float)(gn / sgm0[s]) : 0.f;
        isg[s] = 1.f;
        in2[s] = (float)(kInnerRtol * kInnerRtol);
      }
    }
    __syncthreads();
    const float rtol2f = (float)(rtol * rtol);
#pragma unroll
    for (int s = 0; s < SGP; ++s) {
      bad[s] = s < kv && !(isfinite(nrm[s]) && isfinite(nrm[SGP + s]));
      done[s] = s >= kv || (!bad[s] && !(nrm[s] > 0.0));
      act[s] = !done[s] && !bad[s];
      its[s] = 0;
    }
    float r[VPT][SGP], q[VPT][SGP], d[VPT][SGP];
    int32_t it = 0;
    bool first = true;
    while (it < max_iter) {
      if (!first) {  // FP64 residual of the current iterates, normalised into FP32
        __syncthreads();
        float acc[2 * SGP];
#pragma unroll
        for (int s = 0; s < 2 * SGP; ++s) acc[s] = 0.f;
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          const int32_t v = threadIdx.x + k * NT;
          if (v < nv) {
            double res[SGP];
            const int32_t ov = ord.perm[v];
            group_residual<SGP>(v, ov, g.vptr[ov], nv, vp, NO, D, O, X, gl, act, res);
#pragma unroll
            for (int s = 0; s < SGP; ++s) {
              float rs = 0.f;
              if (act[s]) {
                const float ri = (float)(res[s] * igd[s]);
                rs = ri * Ds[v] * cgs[s];
                acc[s] = fmaf(ri, ri, acc[s]);
                acc[SGP + s] = fmaf(rs, rs, acc[SGP + s]);
              }
              r[k][s] = rs;
            }
          }
        }
        group_sum<NT, 2 * SGP>(acc, shw[0]);
#pragma unroll
        for (int s = 0; s < SGP; ++s) {
          if (!act[s]) continue;
          if (!isfinite(acc[s]) || !isfinite(acc[SGP + s])) {
            bad[s] = true;
            act[s] = false;
          } else if (acc[s] <= rtol2f) {
            done[s] = true;
            act[s] = false;
          }
        }
        __syncthreads();  // every thread is done with isg / sgm of the last step
        if (threadIdx.x == 0) {
#pragma unroll
          for (int s = 0; s < SGP; ++s) {
            if (act[s]) {
              const double ratio = sqrt((double)acc[SGP + s]);  // sigma / sigma0
              sgm[s] = sgm0[s] * ratio;
              isg[s] = (float)(1.0 / ratio);
              // solve the correction only as far as this step needs (a tenth
              // of the remaining ratio), never tighter than the FP32 floor
              const double need = 0.1 * rtol / sqrt((double)acc[s]);
              const double e = need > kInnerRtol ? need : kInnerRtol;
              in2[s] = (float)(e * e);
            }
          }
        }
        __syncthreads();
      } else {
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          const int32_t v = threadIdx.x + k * NT;
          const int32_t ov = v < nv ? ord.perm[v] : 0;
#pragma unroll
          for (int s = 0; s < SGP; ++s)
            r[k][s] = (act[s] && v < nv)
                          ? (float)(gl[(int64_t)s * nv + ov] * (double)Ds[v] * isg0[s])
                          : 0.f;
        }
      }
      first = false;
      bool any = false;
#pragma unroll
      for (int s = 0; s < SGP; ++s) any = any || act[s];
      if (!any) break;
      // inner CG on the scaled system from d = 0, right-hand side of unit norm
      float rz[SGP];
#pragma unroll
      for (int s = 0; s < SGP; ++s) rz[s] = 0.f;
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const int32_t v = threadIdx.x + k * NT;
#pragma unroll
        for (int s = 0; s < SGP; ++s) {
          const float rk = act[s] ? r[k][s] * isg[s] : 0.f;
          r[k][s] = rk;
          d[k][s] = 0.f;
          rz[s] += rk * rk;
        }
        if (v < nv) store_row<SGP>(P + (size_t)v * SGP, r[k]);
      }
      group_sum<NT, SGP>(rz, shw[0]);
      bool in[SGP];
      float best[SGP];
      int since[SGP];
      bool anyin = false;
#pragma unroll
      for (int s = 0; s < SGP; ++s) {
        in[s] = act[s] && rz[s] > 0.f && isfinite(rz[s]);
        best[s] = 1.f;
        since[s] = 0;
        anyin = anyin || in[s];
      }
      if (!anyin) break;  // nothing left to reduce in FP32: final test below
      while (it < max_iter) {
        ++it;
#pragma unroll
        for (int s = 0; s < SGP; ++s) its[s] += in[s] ? 1 : 0;
        __syncthreads();  // P from the previous update is visible
        float pq[SGP];
#pragma unroll
        for (int s = 0; s < SGP; ++s) pq[s] = 0.f;
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          const int32_t v = threadIdx.x + k * NT;
          if (v < nv) {
            float acc[SGP], pv[SGP];
            load_row<SGP>(P + (size_t)v * SGP, pv);
#pragma unroll
            for (int s = 0; s < SGP; ++s) acc[s] = pv[s];
            const int32_t kend = vp[v + 1];
            int32_t kk = vp[v];
            for (; kk + 1 < kend; kk += 2) {  // two gathers in flight
              const int2 n0 = NO[kk], n1 = NO[kk + 1];
              float p0[SGP], p1[SGP];
              load_row<SGP>(P + (size_t)n0.x * SGP, p0);
              load_row<SGP>(P + (size_t)n1.x * SGP, p1);
              const float o0 = __int_as_float(n0.y), o1 = __int_as_float(n1.y);
#pragma unroll
              for (int s = 0; s < SGP; ++s) acc[s] = fmaf(o1, p1[s], fmaf(o0, p0[s], acc[s]));
            }
            if (kk < kend) {
              const int2 n0 = NO[kk];
              float p0[SGP];
              load_row<SGP>(P + (size_t)n0.x * SGP, p0);
              const float o0 = __int_as_float(n0.y);
#pragma unroll
              for (int s = 0; s < SGP; ++s) acc[s] = fmaf(o0, p0[s], acc[s]);
            }
#pragma unroll
            for (int s = 0; s < SGP; ++s) {
              q[k][s] = acc[s];
              pq[s] = fmaf(pv[s], acc[s], pq[s]);
            }
          }
        }
        group_sum<NT, SGP>(pq, shw[0]);
        float al[SGP];
#pragma unroll
        for (int s = 0; s < SGP; ++s) {
          al[s] = 0.f;
          if (!in[s]) continue;
          if (!isfinite(pq[s])) {
            bad[s] = true;
            act[s] = false;
            in[s] = false;
          } else if (!(pq[s] > 0.f)) {
            in[s] = false;  // p vanished at the FP32 floor: refine
          } else {
            al[s] = __fdividef(rz[s], pq[s]);
          }
        }
        float rr[SGP];
#pragma unroll
        for (int s = 0; s < SGP; ++s) rr[s] = 0.f;
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          const int32_t v = threadIdx.x + k * NT;
          if (v < nv) {
            float pv[SGP];
            load_row<SGP>(P + (size_t)v * SGP, pv);
#pragma unroll
            for (int s = 0; s < SGP; ++s) {
              d[k][s] = fmaf(al[s], pv[s], d[k][s]);
              r[k][s] = fmaf(-al[s], q[k][s], r[k][s]);
              rr[s] = fmaf(r[k][s], r[k][s], rr[s]);
            }
          }
        }
        group_sum<NT, SGP>(rr, shw[1]);
        float be[SGP];
        bool still = false;
#pragma unroll
        for (int s = 0; s < SGP; ++s) {
          be[s] = 0.f;
          if (!in[s]) continue;
          if (!isfinite(rr[s])) {
            bad[s] = true;
            act[s] = false;
            in[s] = false;
          } else if (rr[s] <= in2[s]) {
            in[s] = false;
          } else {
            if (rr[s] < 0.98f * best[s]) {
              best[s] = rr[s];
              since[s] = 0;
            } else if (++since[s] >= 32) {
              in[s] = false;  // the FP32 recurrence reached its rounding floor
            }
            be[s] = __fdividef(rr[s], rz[s]);
            rz[s] = rr[s];
          }
          still = still || in[s];
        }
        if (!still) break;
        // P = r + beta P for the samples still iterating (own rows only)
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          const int32_t v = threadIdx.x + k * NT;
          if (v < nv) {
            float pv[SGP];
            load_row<SGP>(P + (size_t)v * SGP, pv);
#pragma unroll
            for (int s = 0; s < SGP; ++s)
              if (in[s]) pv[s] = fmaf(be[s], pv[s], r[k][s]);
            store_row<SGP>(P + (size_t)v * SGP, pv);
          }
        }
      }
      // x += sigma D^-1/2 d for the samples of this refinement step
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const int32_t v = threadIdx.x + k * NT;
        if (v < nv) {
#pragma unroll
          for (int s = 0; s < SGP; ++s)
            if (act[s])
              X[(size_t)v * SGP + s] = fma(sgm[s], (double)(Ds[v] * d[k][s]), X[(size_t)v * SGP + s]);
        }
      }
    }
    // iteration budget spent or nothing left to reduce: FP64 test of the final iterates
    bool pending = false;
#pragma unroll
    for (int s = 0; s < SGP; ++s) pending = pending || act[s];
    if (pending) {
      __syncthreads();
      float acc[2 * SGP];
#pragma unroll
      for (int s = 0; s < 2 * SGP; ++s) acc[s] = 0.f;
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const int32_t v = threadIdx.x + k * NT;
        if (v < nv) {
          double res[SGP];
          const int32_t ov = ord.perm[v];
          group_residual<SGP>(v, ov, g.vptr[ov], nv, vp, NO, D, O, X, gl, act, res);
#pragma unroll
          for (int s = 0; s < SGP; ++s) {
            if (act[s]) {
              const float ri = (float)(res[s] * igd[s]);
              acc[s] = fmaf(ri, ri, acc[s]);
            }
          }
        }
      }
      group_sum<NT, 2 * SGP>(acc, shw[0]);
#pragma unroll
      for (int s = 0; s < SGP; ++s)
        if (act[s]) done[s] = acc[s] <= rtol2f;
    }
    // the group's solutions out of shared memory
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const int32_t v = threadIdx.x + k * NT;
      if (v < nv) {
        const int32_t ov = ord.perm[v];
#pragma unroll
        for (int s = 0; s < SGP; ++s)
          if (s < kv) xl[(int64_t)s * nv + ov] = X[(size_t)v * SGP + s];
      }
    }
    if (threadIdx.x == 0) {
      for (int s = 0; s < kv; ++s) {
        iters[l * S + s0 + s] = its[s];
        atomicAdd(&status->iters_total, (unsigned long long)its[s]);
        atomicMax(&status->iters_max, its[s]);
        if (bad[s]) atomicAdd(&status->numeric_flag, 1);
        else if (!done[s]) atomicAdd(&status->n_unconverged, 1);
      }
    }
  }
}

// Shared memory of the preconditioned group kernel: P, R (and Y for the
// learned form) [nv][SGP], Ot and pn [2E], Ds and pc [nv], incidence offsets.
template <int SGP, int PRE>
__host__ __device__ inline size_t group_pre_bytes(int32_t nv, int32_t ne) {
  const size_t vecs = PRE == kPreLearned ? 3 : 2;
  return 4 * ((size_t)nv * SGP * vecs + 4 * (size_t)ne + 3 * (size_t)nv + 1) + 16;
}

// The sample-group PCG with a sparse preconditioner on the Jacobi-scaled
// system: PRE = kPreNeumann (z = pc r + N r, one sweep over the incidences) or
// kPreLearned (z = B B^T r, two sweeps). The residuals of the group are shared
// (R) because the preconditioner reads the neighbours' values. A sample whose
// preconditioner breaks down (r.z <= 0, p.Sp <= 0, non-finite) drops that
// step's correction and continues with Jacobi (z = r) from its last refined
// iterate. Otherwise as pcg_group_kernel.
template <int NT, int VPT, int SGP, int PRE>
__global__ void __launch_bounds__(NT) pcg_group_pre_kernel(
    DevGraph g, int32_t L, int64_t S, const double* __restrict__ diag,
    const double* __restrict__ offv, const float* __restrict__ dscale_t,
    const float* __restrict__ offv_t, const float* __restrict__ pcoef,
    const float* __restrict__ ncoef, const double* __restrict__ gvec,
    double* __restrict__ xout, double rtol, int32_t max_iter, int32_t* __restrict__ iters,
    PcgStatus* status) {
  static_assert(SGP == 2 || SGP == 4, "sample groups of 2 or 4");
  constexpr bool kLearned = PRE == kPreLearned;
  __shared__ __align__(16) float shw[2][(NT / 32) * 2 * SGP];
  __shared__ double shd[(NT / 32 + 1) * 2 * SGP];
  __shared__ double igd[SGP], sgm0[SGP], isg0[SGP], sgm[SGP];
  __shared__ float cgs[SGP], isg[SGP], in2[SGP];
  extern __shared__ __align__(16) unsigned char grp_sm[];
  const int32_t nv = g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  float* P = reinterpret_cast<float*>(grp_sm);    // [nv][SGP]
  float* R = P + (size_t)nv * SGP;                // [nv][SGP]
  float* Y = R + (size_t)nv * SGP;                // [nv][SGP] (learned only)
  float* Ot = kLearned ? Y + (size_t)nv * SGP : Y;  // [2E]
  float* Pn = Ot + ne2;                           // [2E]
  float* Ds = Pn + ne2;                           // [nv]
  float* Pc = Ds + nv;                            // [nv]
  int32_t* vp = reinterpret_cast<int32_t*>(Pc + nv);  // [nv + 1]
  for (int32_t v = threadIdx.x; v <= nv; v += NT) vp[v] = g.vptr[v];
  const int64_t ngrp = (S + SGP - 1) / SGP;
  const int64_t units = (int64_t)L * ngrp;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    // nodes from the largest shift down: the nodes that need the most
    // iterations start first, so the last wave is made of short solves
    const int64_t l = L - 1 - u / ngrp;
    const int64_t s0 = (u % ngrp) * SGP;
    const int kv = (int)(S - s0 < SGP ? S - s0 : SGP);
    __syncthreads();  // the previous unit is done with the shared arrays
    for (int64_t k = threadIdx.x; k < ne2; k += NT) {
      Ot[k] = offv_t[l * ne2 + k];
      Pn[k] = ncoef[l * ne2 + k];
    }
    for (int32_t v = threadIdx.x; v < nv; v += NT) {
      Ds[v] = dscale_t[l * nv + v];
      Pc[v] = pcoef[l * nv + v];
    }
    __syncthreads();
    const double* D = diag + l * nv;
    const double* O = offv + l * ne2;
    const double* gl = gvec + (l * S + s0) * nv;
    double* xl = xout + (l * S + s0) * nv;
    double nrm[2 * SGP];
#pragma unroll
    for (int s = 0; s < 2 * SGP; ++s) nrm[s] = 0.0;
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const int32_t v = threadIdx.x + k * NT;
      if (v < nv) {
#pragma unroll
        for (int s = 0; s < SGP; ++s) {
          if (s < kv) {
            const double gv = gl[(int64_t)s * nv + v];
            const double sv = gv * (double)Ds[v];
            nrm[s] += gv * gv;
            nrm[SGP + s] += sv * sv;
            xl[(int64_t)s * nv + v] = 0.0;
          }
        }
      }
    }
    block_sum<NT, 2 * SGP>(nrm, shd);
    bool act[SGP], done[SGP], bad[SGP], pre_on[SGP];
    int32_t its[SGP], nfb = 0;
    if (threadIdx.x == 0) {
#pragma unroll
      for (int s = 0; s < SGP; ++s) {
        const double gn = sqrt(nrm[s]);
        sgm0[s] = sqrt(nrm[SGP + s]);
        isg0[s] = sgm0[s] > 0.0 ? 1.0 / sgm0[s] : 0.0;
        sgm[s] = sgm0[s];
        igd[s] = gn > 0.0 ? 1.0 / gn : 0.0;
        cgs[s] = sgm0[s] > 0.0 ? (float)(gn / sgm0[s]) : 0.f;
        isg[s] = 1.f;
        in2[s] = (float)(kInnerRtol * kInnerRtol);
      }
    }
    __syncthreads();
    const float rtol2f = (float)(rtol * rtol);
#pragma unroll
    for (int s = 0; s < SGP; ++s) {
      bad[s] = s < kv && !(isfinite(nrm[s]) && isfinite(nrm[SGP + s]));
      done[s] = s >= kv || (!bad[s] && !(nrm[s] > 0.0));
      act[s] = !done[s] && !bad[s];
      pre_on[s] = true;
      its[s] = 0;
    }
    float r[VPT][SGP], q[VPT][SGP], d[VPT][SGP];
    int32_t it = 0;
    bool first = true;
    while (it < max_iter) {
      if (!first) {
        __syncthreads();
        float acc[2 * SGP];
#pragma unroll
        for (int s = 0; s < 2 * SGP; ++s) acc[s] = 0.f;
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          const int32_t v = threadIdx.x + k * NT;
          if (v < nv) {
#pragma unroll
            for (int s = 0; s < SGP; ++s) {
              float rs = 0.f;
              if (act[s]) {
                const double* xs = xl + (int64_t)s * nv;
                double y = D[v] * xs[v];
                for (int32_t kk = vp[v]; kk < vp[v + 1]; ++kk) y += O[kk] * xs[g.adj_nbr[kk]];
                const float ri = (float)((gl[(int64_t)s * nv + v] - y) * igd[s]);
                rs = ri * Ds[v] * cgs[s];
                acc[s] = fmaf(ri, ri, acc[s]);
                acc[SGP + s] = fmaf(rs, rs, acc[SGP + s]);
              }
              r[k][s] = rs;
            }
          }
        }
        group_sum<NT, 2 * SGP>(acc, shw[0]);
#pragma unroll
        for (int s = 0; s < SGP; ++s) {
          if (!act[s]) continue;
          if (!isfinite(acc[s]) || !isfinite(acc[SGP + s])) {
            bad[s] = true;
            act[s] = false;
          } else if (acc[s] <= rtol2f) {
            done[s] = true;
            act[s] = false;
          }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
          for (int s = 0; s < SGP; ++s) {
            if (act[s]) {
              const double ratio = sqrt((double)acc[SGP + s]);
              sgm[s] = sgm0[s] * ratio;
              isg[s] = (float)(1.0 / ratio);
              const double need = 0.1 * rtol / sqrt((double)acc[s]);
              const double e = need > kInnerRtol ? need : kInnerRtol;
              in2[s] = (float)(e * e);
            }
          }
        }
        __syncthreads();
      } else {
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          const int32_t v = threadIdx.x + k * NT;
#pragma unroll
          for (int s = 0; s < SGP; ++s)
            r[k][s] = (act[s] && v < nv)
                          ? (float)(gl[(int64_t)s * nv + v] * (double)Ds[v] * isg0[s])
                          : 0.f;
        }
      }
      first = false;
      bool any = false;
#pragma unroll
      for (int s = 0; s < SGP; ++s) any = any || act[s];
      if (!any) break;
      // inner start: r (unit scaled residual) shared, z = P r, p = z
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const int32_t v = threadIdx.x + k * NT;
#pragma unroll
        for (int s = 0; s < SGP; ++s) {
          r[k][s] = act[s] ? r[k][s] * isg[s] : 0.f;
          d[k][s] = 0.f;
        }
        if (v < nv) store_row<SGP>(R + (size_t)v * SGP, r[k]);
      }
      float rz[2 * SGP];  // r.z, then r.r
      prec_group_apply<NT, VPT, SGP, kLearned>(g, nv, vp, Pc, Pn, R, Y, r, pre_on, q, rz);
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const int32_t v = threadIdx.x + k * NT;
        if (v < nv) store_row<SGP>(P + (size_t)v * SGP, q[k]);
      }
      group_sum<NT, 2 * SGP>(rz, shw[1]);
      bool in[SGP], drop[SGP];
      float best[SGP], rrv[SGP];
      int since[SGP];
      bool anyin = false;
#pragma unroll
      for (int s = 0; s < SGP; ++s) {
        drop[s] = false;
        rrv[s] = rz[SGP + s];
        in[s] = act[s] && rz[SGP + s] > 0.f && isfinite(rz[SGP + s]);
        if (in[s] && pre_on[s] && !(rz[s] > 0.f && isfinite(rz[s]))) {
          pre_on[s] = false;  // breakdown at the start: Jacobi from here on
          ++nfb;
          in[s] = false;
          drop[s] = true;
        }
        best[s] = 1.f;
        since[s] = 0;
        anyin = anyin || in[s];
      }
      bool restart = false;
#pragma unroll
      for (int s = 0; s < SGP; ++s) restart = restart || (drop[s] && act[s]);
      if (!anyin && !restart) break;
      while (anyin && it < max_iter) {
        ++it;
#pragma unroll
        for (int s = 0; s < SGP; ++s) its[s] += in[s] ? 1 : 0;
        __syncthreads();  // P visible
        float pq[SGP];
#pragma unroll
        for (int s = 0; s < SGP; ++s) pq[s] = 0.f;
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          const int32_t v = threadIdx.x + k * NT;
          if (v < nv) {
            float acc[SGP], pv[SGP];
            load_row<SGP>(P + (size_t)v * SGP, pv);
#pragma unroll
            for (int s = 0; s < SGP; ++s) acc[s] = pv[s];
            const int32_t kend = vp[v + 1];
            for (int32_t kk = vp[v]; kk < kend; ++kk) {
              const float o = Ot[kk];
              float pw[SGP];
              load_row<SGP>(P + (size_t)g.adj_nbr[kk] * SGP, pw);
#pragma unroll
              for (int s = 0; s < SGP; ++s) acc[s] = fmaf(o, pw[s], acc[s]);
            }
#pragma unroll
            for (int s = 0; s < SGP; ++s) {
              q[k][s] = acc[s];
              pq[s] = fmaf(pv[s], acc[s], pq[s]);
            }
          }
        }
        group_sum<NT, SGP>(pq, shw[0]);
        float al[SGP];
#pragma unroll
        for (int s = 0; s < SGP; ++s) {
          al[s] = 0.f;
          if (!in[s]) continue;
          if (!isfinite(pq[s]) || !(pq[s] > 0.f)) {
            in[s] = false;
            // p vanishing next to an FP32-small residual is the rounding floor;
            // otherwise the preconditioner broke down
            if (pre_on[s] && (!isfinite(pq[s]) || rrv[s] > 1e-10f)) {
              pre_on[s] = false;
              ++nfb;
              drop[s] = true;
            } else if (!isfinite(pq[s])) {
              bad[s] = true;
              act[s] = false;
            }
          } else {
            al[s] = __fdividef(rz[s], pq[s]);
          }
        }
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          const int32_t v = threadIdx.x + k * NT;
          if (v < nv) {
            float pv[SGP];
            load_row<SGP>(P + (size_t)v * SGP, pv);
#pragma unroll
            for (int s = 0; s < SGP; ++s) {
              d[k][s] = fmaf(al[s], pv[s], d[k][s]);
              r[k][s] = fmaf(-al[s], q[k][s], r[k][s]);
            }
            store_row<SGP>(R + (size_t)v * SGP, r[k]);
          }
        }
        float rzn[2 * SGP];
        prec_group_apply<NT, VPT, SGP, kLearned>(g, nv, vp, Pc, Pn, R, Y, r, pre_on, q, rzn);
        group_sum<NT, 2 * SGP>(rzn, shw[1]);
        float be[SGP];
        bool still = false;
#pragma unroll
        for (int s = 0; s < SGP; ++s) {
          be[s] = 0.f;
          if (!in[s]) continue;
          const float rr = rzn[SGP + s];
          if (!isfinite(rr)) {
            bad[s] = true;
            act[s] = false;
            in[s] = false;
          } else if (rr <= in2[s]) {
            in[s] = false;  // converged (r.z may have lost its sign at this size)
          } else if (pre_on[s] && !(rzn[s] > 0.f && isfinite(rzn[s]))) {
            in[s] = false;  // breakdown: drop this step's correction
            pre_on[s] = false;
            ++nfb;
            drop[s] = true;
          } else {
            if (rr < 0.98f * best[s]) {
              best[s] = rr;
              since[s] = 0;
            } else if (++since[s] >= 32) {
              in[s] = false;
            }
            be[s] = __fdividef(rzn[s], rz[s]);
            rz[s] = rzn[s];
          }
          rrv[s] = rr;
          still = still || in[s];
        }
        if (!still) break;
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
          const int32_t v = threadIdx.x + k * NT;
          if (v < nv) {
            float pv[SGP];
            load_row<SGP>(P + (size_t)v * SGP, pv);
#pragma unroll
            for (int s = 0; s < SGP; ++s)
              if (in[s]) pv[s] = fmaf(be[s], pv[s], q[k][s]);
            store_row<SGP>(P + (size_t)v * SGP, pv);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const int32_t v = threadIdx.x + k * NT;
        if (v < nv) {
#pragma unroll
          for (int s = 0; s < SGP; ++s)
            if (act[s] && !drop[s])
              xl[(int64_t)s * nv + v] = fma(sgm[s], (double)(Ds[v] * d[k][s]), xl[(int64_t)s * nv + v]);
        }
      }
    }
    bool pending = false;
#pragma unroll
    for (int s = 0; s < SGP; ++s) pending = pending || act[s];
    if (pending) {
      __syncthreads();
      float acc[2 * SGP];
#pragma unroll
      for (int s = 0; s < 2 * SGP; ++s) acc[s] = 0.f;
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const int32_t v = threadIdx.x + k * NT;
        if (v < nv) {
#pragma unroll
          for (int s = 0; s < SGP; ++s) {
            if (act[s]) {
              const double* xs = xl + (int64_t)s * nv;
              double y = D[v] * xs[v];
              for (int32_t kk = vp[v]; kk < vp[v + 1]; ++kk) y += O[kk] * xs[g.adj_nbr[kk]];
              const float ri = (float)((gl[(int64_t)s * nv + v] - y) * igd[s]);
              acc[s] = fmaf(ri, ri, acc[s]);
            }
          }
        }
      }
      group_sum<NT, 2 * SGP>(acc, shw[0]);
#pragma unroll
      for (int s = 0; s < SGP; ++s)
        if (act[s]) done[s] = acc[s] <= rtol2f;
    }
    if (threadIdx.x == 0) {
      for (int s = 0; s < kv; ++s) {
        iters[l * S + s0 + s] = its[s];
        atomicAdd(&status->iters_total, (unsigned long long)its[s]);
        atomicMax(&status->iters_max, its[s]);
        if (!pre_on[s]) atomicAdd(&status->n_fallback, 1);
        if (bad[s]) atomicAdd(&status->numeric_flag, 1);
        else if (!done[s]) atomicAdd(&status->n_unconverged, 1);
      }
    }
    (void)nfb;
  }
}

template <int NT, int VPT, int SGP, int PRE>
void launch_group_pre(const DevGraph& g, int32_t L, int64_t S, const double* diag,
                      const double* offv, const float* dscale_t, const float* offv_t,
                      const float* pc, const float* pn, const double* gvec, double* x,
                      double rtol, int32_t max_iter, int32_t* iters, PcgStatus* status,
                      cudaStream_t st) {
  const size_t dyn = group_pre_bytes<SGP, PRE>(g.nv, g.ne);
  cudaFuncSetAttribute(pcg_group_pre_kernel<NT, VPT, SGP, PRE>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  const int64_t units = (int64_t)L * ((S + SGP - 1) / SGP);
  const int blocks = (int)(units < sm_count() * 8 ? units : sm_count() * 8);
  pcg_group_pre_kernel<NT, VPT, SGP, PRE><<<blocks, NT, dyn, st>>>(
      g, L, S, diag, offv, dscale_t, offv_t, pc, pn, gvec, x, rtol, max_iter, iters, status);
}

bool group_pre_fits(const DevGraph& g, int pre) {
  const int sgp = g.nv <= 4 * kThreadsG ? 4 : 2;
  size_t dyn;
  if (pre == kPreLearned)
    dyn = sgp == 4 ? group_pre_bytes<4, kPreLearned>(g.nv, g.ne)
                   : group_pre_bytes<2, kPreLearned>(g.nv, g.ne);
  else
    dyn = sgp == 4 ? group_pre_bytes<4, kPreNeumann>(g.nv, g.ne)
                   : group_pre_bytes<2, kPreNeumann>(g.nv, g.ne);
  return g.nv <= 8 * kThreadsG && dyn + 8 * 1024 <= kSmemMax;
}

template <int NT, int VPT, int SGP>
void launch_group(const DevGraph& g, const VertexOrder& ord, int32_t L, int64_t S,
                  const double* diag, const double* offv, const float* dscale_t,
                  const float* offv_t, const double* gvec, double* x,
                  double rtol, int32_t max_iter, int32_t* iters, PcgStatus* status,
                  cudaStream_t st) {
  const size_t dyn = group_bytes<SGP>(g.nv, g.ne);
  cudaFuncSetAttribute(pcg_group_kernel<NT, VPT, SGP>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  const int64_t units = (int64_t)L * ((S + SGP - 1) / SGP);
  const int blocks = (int)(units < sm_count() * 8 ? units : sm_count() * 8);
  pcg_group_kernel<NT, VPT, SGP><<<blocks, NT, dyn, st>>>(
      g, ord, L, S, diag, offv, dscale_t, offv_t, gvec, x, rtol, max_iter, iters, status);
}

// The group layout applies when every vertex fits the per-thread register
// arrays and the node's data fits shared memory.
bool group_fits(const DevGraph& g) {
  const int sgp = g.nv <= 4 * kThreadsG ? 4 : 2;
  const size_t dyn = sgp == 4 ? group_bytes<4>(g.nv, g.ne) : group_bytes<2>(g.nv, g.ne);
  return g.nv <= 8 * kThreadsG && dyn + 8 * 1024 <= kSmemMax;
}

}  // namespace

bool pcg_batch_selected(const DevGraph& g, int layout, int pre) {
  if (pre != kPreJacobi) return false;
  if (layout == 4) return true;
  if ((layout == 2 || layout == 3) && group_fits(g)) return false;
  return layout != 1;
}

template <typename VT>
void launch_pcg(const DevGraph& g, const VertexOrder& ord, const int4* ell, int32_t L, int64_t S,
                const double* diag, const double* offv, const VT* dscale_t, const VT* offv_t, int pre, const VT* pc, const VT* pn,
                const double* gvec, double* x, VT* d, VT* r, VT* p, VT* q, VT* y, double rtol,
                int32_t max_iter, int32_t* iters, PcgStatus* status, int layout,
                cudaStream_t st, const PcgPairs* pairs) {
  const int64_t nsys = (int64_t)L * S;
  if constexpr (sizeof(VT) == 4) {
    if (layout == 4 && pre == kPreJacobi && pairs) {
      launch_pcg_batch(g, ell, L, S, diag, offv, dscale_t, offv_t, gvec, x, r, p, q, d, *pairs,
                       rtol, max_iter, iters, status, st);
      return;
    }
    if ((layout == 2 || layout == 3) && pre == kPreJacobi && group_fits(g)) {
#define GRF_GROUP(NT, VPT, SGP)                                                               \
  launch_group<NT, VPT, SGP>(g, ord, L, S, diag, offv, dscale_t, offv_t, gvec, x, rtol,      \
                             max_iter, iters, status, st)
      if (layout == 2) {  // 512 threads, groups of 4 samples
        if (g.nv <= kThreadsG) GRF_GROUP(512, 1, 4);
        else if (g.nv <= 2 * kThreadsG) GRF_GROUP(512, 2, 4);
        else if (g.nv <= 4 * kThreadsG) GRF_GROUP(512, 4, 4);
        else GRF_GROUP(512, 8, 2);
      } else {  // 256 threads, groups of 2 samples: more resident CTAs per SM
        if (g.nv <= 256) GRF_GROUP(256, 1, 2);
        else if (g.nv <= 512) GRF_GROUP(256, 2, 2);
        else if (g.nv <= 1024) GRF_GROUP(256, 4, 2);
        else if (g.nv <= 2048) GRF_GROUP(256, 8, 2);
        else GRF_GROUP(512, 8, 2);
      }
#undef GRF_GROUP
      return;
    }
    if ((layout == 2 || layout == 3) && pre != kPreJacobi && group_pre_fits(g, pre)) {
#define GRF_GROUP_PRE(VPT, SGP, PRE)                                                          \
  launch_group_pre<512, VPT, SGP, PRE>(g, L, S, diag, offv, dscale_t, offv_t, pc, pn, gvec, x, \
                                       rtol, max_iter, iters, status, st)
#define GRF_GROUP_PRE_ALL(PRE)                                                 \
  if (g.nv <= kThreadsG) GRF_GROUP_PRE(1, 4, PRE);                             \
  else if (g.nv <= 2 * kThreadsG) GRF_GROUP_PRE(2, 4, PRE);                    \
  else if (g.nv <= 4 * kThreadsG) GRF_GROUP_PRE(4, 4, PRE);                    \
  else GRF_GROUP_PRE(8, 2, PRE);
      if (pre == kPreLearned) {
        GRF_GROUP_PRE_ALL(kPreLearned)
      } else {
        GRF_GROUP_PRE_ALL(kPreNeumann)
      }
#undef GRF_GROUP_PRE_ALL
#undef GRF_GROUP_PRE
      return;
    }
  }
  if constexpr (sizeof(VT) == 4) {
    // larger graphs: samples batched in rows of 8 (the vectors are carved with
    // the sample count padded to a multiple of 8)
    if (layout != 1 && pre == kPreJacobi && pairs) {
      launch_pcg_batch(g, ell, L, S, diag, offv, dscale_t, offv_t, gvec, x, r, p, q, d, *pairs,
                       rtol, max_iter, iters, status, st);
      return;
    }
  }
  int blocks = (int)(nsys < sm_count() * 16 ? nsys : sm_count() * 16);
  if (blocks < 1) blocks = 1;
  const size_t smem = (sizeof(VT) == 4 ? sizeof(double) : 0) * (size_t)g.nv +
                      (pre == kPreLearned ? 5 : 4) * sizeof(VT) * (size_t)g.nv;
  if (smem <= kSmemMax - 16 * 1024) {
    // dynamic + static may pass the 48 KB default; per device: set at every launch
    cudaFuncSetAttribute(pcg_kernel<VT, true, kThreadsA>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pcg_kernel<VT, true, kThreadsA><<<blocks, kThreadsA, smem, st>>>(
        g, L, S, diag, offv, dscale_t, offv_t, pre, pc, pn, gvec, x, d, r, p, q, y, rtol, max_iter,
        iters, status);
  } else {
    constexpr int kNT = kThreadsL;
    int gb = (int)(nsys < sm_count() * (2048 / kNT) * 2 ? nsys : sm_count() * (2048 / kNT) * 2);
    if (gb < 1) gb = 1;
    pcg_kernel<VT, false, kNT><<<gb, kNT, 0, st>>>(g, L, S, diag, offv, dscale_t, offv_t, pre, pc,
                                                  pn, gvec, x, d, r, p, q, y, rtol, max_iter,
                                                  iters, status);
  }
}
#define GRF_INST(VT)                                                                          \
  template void launch_pcg<VT>(const DevGraph&, const VertexOrder&, const int4*, int32_t,  \
                               int64_t,                                                      \
                               const double*, const double*, const VT*, const VT*, int,      \
                               const VT*, const VT*, const double*, double*, VT*, VT*, VT*,  \
                               VT*, VT*, double, int32_t, int32_t*, PcgStatus*, int,         \
                               cudaStream_t, const PcgPairs*);
GRF_INST(float)
GRF_INST(double)
#undef GRF_INST

}  // namespace grf
