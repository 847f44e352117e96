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
// the stopping test is always on the FP64 residual. Dot products are FP32
// partial sums over one thread's vertices, combined across the block in FP64.
// On GB300 FP64 arithmetic runs at a small fraction of the FP32 rate, which is
// what this split is for.
//
// One CTA owns one system for its whole life: the reductions are CTA-local
// (warp shuffles + shared memory), so no CTA ever waits on another and every
// loop is bounded by max_iter. When the system's vectors fit, they live in
// shared memory.
#include "grf_internal.h"

namespace grf {
namespace {

constexpr int kThreads = 256;
constexpr size_t kSmemVectorsMax = 200 * 1024;
constexpr double kInnerRtol = 1e-4;

template <int N>
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

// Per-system vectors: VT d (update), r, p, q; FP64 x (the iterate) when refining.
template <typename VT>
struct SysVecs {
  VT *d, *r, *p, *q;
  double* x;
};

// FP64 residual r_i = g_i - (S x)_i
__device__ __forceinline__ double residual(const DevGraph& g, const double* D, const double* O,
                                           const double* gs, const double* x, int32_t i) {
  double y = D[i] * x[i];
  for (int32_t k = g.vptr[i]; k < g.vptr[i + 1]; ++k) y += O[k] * x[g.adj_nbr[k]];
  return gs[i] - y;
}

// dscale: FP64 mode 1 / D; mixed mode 1 / sqrt(D).
// offv_t: FP64 mode the blocks; mixed mode the Jacobi-scaled blocks.
template <typename VT, bool kSmem>
__global__ void __launch_bounds__(kThreads) pcg_kernel(
    DevGraph g, int32_t L, int64_t S, const double* __restrict__ diag,
    const double* __restrict__ offv, const VT* __restrict__ dscale_t,
    const VT* __restrict__ offv_t, const double* __restrict__ gvec, double* __restrict__ xout,
    VT* __restrict__ gd, VT* __restrict__ gr, VT* __restrict__ gp, VT* __restrict__ gq,
    double rtol, int32_t max_iter, int32_t* __restrict__ iters, PcgStatus* status) {
  constexpr bool kRefine = sizeof(VT) == 4;
  __shared__ double sh[(kThreads / 32) * 2];
  extern __shared__ __align__(16) unsigned char vec_sm[];
  const int64_t nsys = (int64_t)L * S;
  const int32_t nv = g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  for (int64_t sys = blockIdx.x; sys < nsys; sys += gridDim.x) {
    const int64_t l = sys / S;
    const double* D = diag + l * nv;
    const double* O = offv + l * ne2;
    const VT* Ds = dscale_t + l * nv;
    const VT* Ot = offv_t + l * ne2;
    const double* gs = gvec + sys * nv;
    double* xo = xout + sys * nv;
    SysVecs<VT> v;
    if (kSmem) {
      v.x = reinterpret_cast<double*>(vec_sm);
      VT* base = reinterpret_cast<VT*>(vec_sm + (kRefine ? sizeof(double) * nv : 0));
      v.d = base;
      v.r = base + nv;
      v.p = base + 2 * (int64_t)nv;
      v.q = base + 3 * (int64_t)nv;
    } else {
      v.x = xo;
      v.d = gd + sys * nv;
      v.r = gr + sys * nv;
      v.p = gp + sys * nv;
      v.q = gq + sys * nv;
    }
    // FP64 mode: one PCG run on d (= u, since it starts from 0).
    // Mixed mode: x (FP64) accumulates the scaled FP32 updates of each step.
    double gg[2] = {0.0, 0.0};
    for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
      const double gv = gs[i];
      gg[0] += gv * gv;
      if (kRefine) {
        const double sv = gv * (double)Ds[i];
        gg[1] += sv * sv;
        v.x[i] = 0.0;
      }
      v.d[i] = (VT)0;
    }
    block_sum<2>(gg, sh);
    const double tol2 = rtol * rtol * gg[0];
    int32_t it = 0;
    bool bad = !isfinite(gg[0]) || !isfinite(gg[1]);
    bool done = bad || !(gg[0] > 0.0);
    double sig2 = gg[1];  // ||D^-1/2 r||^2 of the current refinement step
    while (!done && it < max_iter) {
      double sigma = 1.0;
      if (kRefine) {
        if (it > 0) {  // FP64 residual of the current iterate and its scaled norm
          __syncthreads();
          double acc[2] = {0.0, 0.0};
          for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
            const double ri = residual(g, D, O, gs, v.x, i);
            const double si = ri * (double)Ds[i];
            acc[0] += ri * ri;
            acc[1] += si * si;
          }
          block_sum<2>(acc, sh);
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
          const double ri = it > 0 ? residual(g, D, O, gs, v.x, i) : gs[i];
          v.r[i] = (VT)(ri * (double)Ds[i] * inv);
          v.d[i] = (VT)0;
        }
        __syncthreads();
      } else {
        for (int32_t i = threadIdx.x; i < nv; i += kThreads) v.r[i] = (VT)gs[i];
      }
      // (P)CG on the inner system from d = 0
      VT rz0 = (VT)0;
      for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
        const VT ri = v.r[i];
        const VT z = kRefine ? ri : ri * Ds[i];
        v.p[i] = z;
        rz0 += ri * z;
      }
      double a0[1] = {(double)rz0};
      block_sum<1>(a0, sh);
      double rz = a0[0];
      // inner stop: mixed relative to the unit start, FP64 on the true residual
      const double inner2 = kRefine ? kInnerRtol * kInnerRtol : tol2;
      double best = kRefine ? 1.0 : gg[0];
      int since_best = 0;
      bool inner_done = false;
      while (it < max_iter) {
        ++it;
        __syncthreads();  // p from the previous update is visible
        VT pqf = (VT)0;
        for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
          VT y = kRefine ? v.p[i] : (VT)D[i] * v.p[i];
          for (int32_t k = g.vptr[i]; k < g.vptr[i + 1]; ++k) y += Ot[k] * v.p[g.adj_nbr[k]];
          v.q[i] = y;
          pqf += v.p[i] * y;
        }
        double pq[1] = {(double)pqf};
        block_sum<1>(pq, sh);
        if (!isfinite(pq[0])) {
          bad = true;
          break;
        }
        if (!(pq[0] > 0.0)) {  // p vanished (mixed: at the FP32 floor)
          if (!kRefine) bad = true;
          break;
        }
        const VT af = (VT)(rz / pq[0]);
        VT rzf = (VT)0, rrf = (VT)0;
        for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
          v.d[i] += af * v.p[i];
          const VT ri = v.r[i] - af * v.q[i];
          v.r[i] = ri;
          rzf += kRefine ? ri * ri : ri * ri * Ds[i];
          rrf += ri * ri;
        }
        double a2[2] = {(double)rzf, (double)rrf};
        block_sum<2>(a2, sh);
        if (!isfinite(a2[0])) {
          bad = true;
          break;
        }
        if (a2[1] <= inner2) {
          inner_done = true;
          break;
        }
        if (kRefine) {  // the FP32 recurrence has reached its rounding floor
          if (a2[1] < 0.98 * best) {
            best = a2[1];
            since_best = 0;
          } else if (++since_best >= 32) {
            break;
          }
        }
        const VT bf = (VT)(a2[0] / rz);
        rz = a2[0];
        for (int32_t i = threadIdx.x; i < nv; i += kThreads)
          v.p[i] = (kRefine ? v.r[i] : v.r[i] * Ds[i]) + bf * v.p[i];
      }
      if (bad) break;
      if (!kRefine) {
        done = inner_done;
        break;
      }
      __syncthreads();
      for (int32_t i = threadIdx.x; i < nv; i += kThreads)
        v.x[i] += sigma * (double)Ds[i] * (double)v.d[i];
    }
    if (kRefine && !done && !bad) {
      // iteration budget spent: test the FP64 residual of the final iterate
      __syncthreads();
      double acc[1] = {0.0};
      for (int32_t i = threadIdx.x; i < nv; i += kThreads) {
        const double ri = residual(g, D, O, gs, v.x, i);
        acc[0] += ri * ri;
      }
      block_sum<1>(acc, sh);
      done = acc[0] <= tol2;
    }
    __syncthreads();
    if (kRefine) {
      if (kSmem)
        for (int32_t i = threadIdx.x; i < nv; i += kThreads) xo[i] = v.x[i];
    } else {
      for (int32_t i = threadIdx.x; i < nv; i += kThreads) xo[i] = (double)v.d[i];
    }
    if (threadIdx.x == 0) {
      iters[sys] = it;
      atomicAdd(&status->iters_total, (unsigned long long)it);
      atomicMax(&status->iters_max, it);
      if (bad) atomicAdd(&status->numeric_flag, 1);
      else if (!done) atomicAdd(&status->n_unconverged, 1);
    }
    __syncthreads();
  }
}

}  // namespace

template <typename VT>
void launch_pcg(const DevGraph& g, int32_t L, int64_t S, const double* diag, const double* offv,
                const VT* dscale_t, const VT* offv_t, const double* gvec, double* x, VT* d,
                VT* r, VT* p, VT* q, double rtol, int32_t max_iter, int32_t* iters,
                PcgStatus* status, cudaStream_t st) {
  const int64_t nsys = (int64_t)L * S;
  int blocks = (int)(nsys < 152 * 16 ? nsys : 152 * 16);
  if (blocks < 1) blocks = 1;
  const size_t smem = (sizeof(VT) == 4 ? sizeof(double) : 0) * (size_t)g.nv +
                      4 * sizeof(VT) * (size_t)g.nv;
  if (smem <= kSmemVectorsMax) {
    if (smem > 48 * 1024)  // per device: set at every launch
      cudaFuncSetAttribute(pcg_kernel<VT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    pcg_kernel<VT, true><<<blocks, kThreads, smem, st>>>(g, L, S, diag, offv, dscale_t, offv_t,
                                                         gvec, x, d, r, p, q, rtol, max_iter,
                                                         iters, status);
  } else {
    pcg_kernel<VT, false><<<blocks, kThreads, 0, st>>>(g, L, S, diag, offv, dscale_t, offv_t,
                                                       gvec, x, d, r, p, q, rtol, max_iter, iters,
                                                       status);
  }
}
#define GRF_INST(VT)                                                                          \
  template void launch_pcg<VT>(const DevGraph&, int32_t, int64_t, const double*, const double*, \
                               const VT*, const VT*, const double*, double*, VT*, VT*, VT*, VT*, \
                               double, int32_t, int32_t*, PcgStatus*, cudaStream_t);
GRF_INST(float)
GRF_INST(double)
#undef GRF_INST

}  // namespace grf
