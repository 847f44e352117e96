// Jacobi-preconditioned CG on the vertex Schur systems S^(l) u = g (Eq.
// global_schur; Sec. 3, Phase 4), one system per (node l, sample s).
//
// S^(l) is applied from its per-edge 2x2 blocks: y_v = D_v x_v + sum over the
// incidences k of v of offv_k x_{nbr(k)} (Eq. goal_func_1 with the blocks of
// Eq. local_reduced_schur). Preconditioner z = r / D. Stop when
// ||r||_2 <= rtol ||g||_2 or after max_iter iterations (counted as
// unconverged); a zero right-hand side gives u = 0. Dot products and all
// vectors are FP64.
//
// One CTA owns one system for its whole life: the reductions are CTA-local
// (warp shuffles + shared memory), so no CTA ever waits on another and every
// loop is bounded by max_iter.
#include "grf_internal.h"

namespace grf {
namespace {

constexpr int kThreads = 256;

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

__global__ void __launch_bounds__(kThreads) pcg_jacobi_kernel(
    DevGraph g, int32_t L, int64_t S, const double* __restrict__ diag,
    const double* __restrict__ offv, const double* __restrict__ gvec, double* __restrict__ x,
    double* __restrict__ r, double* __restrict__ p, double* __restrict__ q, double rtol,
    int32_t max_iter, int32_t* __restrict__ iters, PcgStatus* status) {
  __shared__ double sh[(kThreads / 32) * 2];
  const int64_t nsys = (int64_t)L * S;
  const int32_t nv = g.nv;
  for (int64_t sys = blockIdx.x; sys < nsys; sys += gridDim.x) {
    const int64_t l = sys / S;
    const double* D = diag + l * nv;
    const double* O = offv + l * 2 * (int64_t)g.ne;
    const double* gs = gvec + sys * nv;
    double* xs = x + sys * nv;
    double* rs = r + sys * nv;
    double* ps = p + sys * nv;
    double* qs = q + sys * nv;

    double acc[2] = {0.0, 0.0};
    for (int32_t v = threadIdx.x; v < nv; v += kThreads) {
      const double gv = gs[v];
      const double z = gv / D[v];
      xs[v] = 0.0;
      rs[v] = gv;
      ps[v] = z;
      acc[0] += gv * z;
      acc[1] += gv * gv;
    }
    block_sum<2>(acc, sh);
    double rz = acc[0];
    const double tol2 = rtol * rtol * acc[1];
    int32_t it = 0;
    bool done = !(acc[1] > 0.0);
    bool bad = !isfinite(acc[0]) || !isfinite(acc[1]);
    if (bad) done = true;
    while (!done && it < max_iter) {
      ++it;
      __syncthreads();  // p from the previous update is visible
      double pq[1] = {0.0};
      for (int32_t v = threadIdx.x; v < nv; v += kThreads) {
        double y = D[v] * ps[v];
        for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) y += O[k] * ps[g.adj_nbr[k]];
        qs[v] = y;
        pq[0] += ps[v] * y;
      }
      block_sum<1>(pq, sh);
      if (!(pq[0] > 0.0) || !isfinite(pq[0])) {
        bad = true;
        break;
      }
      const double alpha = rz / pq[0];
      double a2[2] = {0.0, 0.0};
      for (int32_t v = threadIdx.x; v < nv; v += kThreads) {
        xs[v] += alpha * ps[v];
        const double rv = rs[v] - alpha * qs[v];
        rs[v] = rv;
        a2[0] += rv * rv / D[v];
        a2[1] += rv * rv;
      }
      block_sum<2>(a2, sh);
      if (!isfinite(a2[0])) {
        bad = true;
        break;
      }
      if (a2[1] <= tol2) {
        done = true;
        break;
      }
      const double beta = a2[0] / rz;
      rz = a2[0];
      for (int32_t v = threadIdx.x; v < nv; v += kThreads) ps[v] = rs[v] / D[v] + beta * ps[v];
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

void launch_pcg_jacobi(const DevGraph& g, int32_t L, int64_t S, const double* diag,
                       const double* offv, const double* gvec, double* x, double* r, double* p,
                       double* q, double rtol, int32_t max_iter, int32_t* iters, PcgStatus* status,
                       cudaStream_t st) {
  int64_t nsys = (int64_t)L * S;
  int blocks = (int)(nsys < 152 * 16 ? nsys : 152 * 16);
  if (blocks < 1) blocks = 1;
  pcg_jacobi_kernel<<<blocks, kThreads, 0, st>>>(g, L, S, diag, offv, gvec, x, r, p, q, rtol,
                                                max_iter, iters, status);
}

}  // namespace grf
