// Per-edge 2x2 Schur blocks of A = alpha M_L + gamma K (Eq. local_reduced_schur)
// and the vertex Schur diagonal (Eq. global_schur), in FP64.
//
// On edge e (h = h_e, n = n_e elements, m = n - 1 interior nodes) the interior
// block is A_II = c T with c = gamma / h and T = tridiag(-1, 2 + delta, -1),
// delta = (alpha / gamma + kappa^2) h^2; the vertex-interior couplings are -c and
// the edge's share of A_vv is c (1 + delta / 2). With 2 + delta = 2 cosh(theta),
// the inverse of T has (T^{-1})_11 = sinh(m theta) / sinh(n theta) and
// (T^{-1})_1m = sinh(theta) / sinh(n theta), so the Schur block is
//   S^(e) = c sinh(theta) [[coth(n theta), -csch(n theta)],
//                          [-csch(n theta), coth(n theta)]]
// (the first entry uses cosh(theta) sinh(n theta) - sinh(m theta) =
// cosh(n theta) sinh(theta)). This is the matrix the paper applies
// matrix-free through one Thomas solve per edge in every PCG iteration
// (Eq. matrix_free_local); it has rank-2 coupling, so the block is exact and
// costs O(1) per (node, edge) instead of O(n_e). sinh(theta) =
// sqrt(delta (1 + delta / 4)) and theta = log1p(delta / 2 + sinh(theta)) avoid
// cancellation for small delta; expm1 keeps large n theta finite.
//
// Consistent mass (the paper's comparison system, Sec. 3 Phase 2 consistent
// case): with a = alpha + gamma kappa^2 the interior block is tridiag(o, d, o),
// d = 2 a h / 3 + 2 gamma / h, o = a h / 6 - gamma / h, the couplings are o and
// the edge's share of A_vv is d / 2. With r = |o| and 2 cosh(theta) = d / r
// (> 2: the block is diagonally dominant) the same algebra gives
//   S^(e) = r sinh(theta) [[coth(n theta), -s csch(n theta)], [..., coth(n theta)]],
// s = 1 for o < 0 and (-1)^n for o > 0 (tridiag(o, d, o) with o > 0 is
// D tridiag(-o, d, -o) D, D = diag((-1)^i)). d / r - 2 is formed without
// cancellation: a h / r for o < 0, (a h / 3 + 4 gamma / h) / r for o > 0.
#include "grf_internal.h"

namespace grf {
namespace {

template <typename T>
__global__ void edge_blocks_kernel(DevGraph g, DevNodes nd, double kappa2, double* __restrict__ saa,
                                   double* __restrict__ sab, SweepParams<T>* __restrict__ prm,
                                   int consistent) {
  const int64_t total = (int64_t)nd.L * g.ne;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = t / g.ne;
    const int32_t e = (int32_t)(t - l * g.ne);
    const double h = g.he[e];
    const double gam = nd.gamma[l];
    double c = gam / h;
    double delta = (nd.alpha[l] / gam + kappa2) * h * h;
    double sgn = 1.0;
    if (consistent) {
      const double a = nd.alpha[l] + gam * kappa2;
      const double o = a * h / 6.0 - gam / h;
      const double r = fabs(o);
      if (!(r > 1e-300)) {  // no coupling through the interior
        const double d2 = a * h / 3.0 + gam / h;
        saa[t] = d2;
        sab[t] = g.nel[e] == 1 ? o : 0.0;
        continue;
      }
      c = r;
      delta = o < 0.0 ? a * h / r : (a * h / 3.0 + 4.0 * gam / h) / r;
      sgn = (o < 0.0 || (g.nel[e] & 1) == 0) ? 1.0 : -1.0;
    }
    // sinh(theta) and theta = acosh(1 + delta/2) = log1p(delta/2 + sinh(theta));
    // with u = expm1(-n theta): exp(-n theta) = 1 + u and
    // 1 - exp(-2 n theta) = -u (2 + u), both free of cancellation
    const double sh = sqrt(delta * (1.0 + 0.25 * delta));
    const double theta = log1p(0.5 * delta + sh);
    const double nth = (double)g.nel[e] * theta;
    const double u = expm1(-nth);
    const double e1 = 1.0 + u;
    const double e2 = -u * (2.0 + u);  // 1 - exp(-2 n theta)
    saa[t] = c * sh * ((2.0 - e2) / e2);
    sab[t] = -sgn * c * sh * (2.0 * e1 / e2);
    if (prm) {
      SweepParams<T> p;
      p.delta = (T)delta;
      p.sc = (T)(nd.weight[l] / c);
      p.sh = (T)sh;
      p.theta = (T)theta;
      prm[t] = p;
    }
  }
}

// diag[l][v] = S_vv, offv in incidence order, and the PCG scaling in precision
// T: 1 / S_vv for FP64 PCG, 1 / sqrt(S_vv) for the Jacobi-scaled FP32 solve.
// x = hi + lo with hi = fl32(x) and lo = fl32(x - hi): 48 of x's 53 bits, the
// form the batched PCG's refinement residual reads the FP64 blocks in.
__device__ __forceinline__ float2 split_pair(double x) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}

template <typename T>
__global__ void vertex_diag_kernel(DevGraph g, int32_t L, const double* __restrict__ saa,
                                   const double* __restrict__ sab, double* __restrict__ diag,
                                   double* __restrict__ offv, T* __restrict__ dscale,
                                   float2* __restrict__ dpair, float2* __restrict__ opair) {
  const int64_t total = (int64_t)L * g.nv;
  const int64_t nadj = 2 * (int64_t)g.ne;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = t / g.nv;
    const int32_t v = (int32_t)(t - l * g.nv);
    double d = 0.0;
    for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
      const int64_t i = l * g.ne + g.adj_edge[k];
      d += saa[i];
      offv[l * nadj + k] = sab[i];
      if (opair) opair[l * nadj + k] = split_pair(sab[i]);
    }
    diag[t] = d;
    if (dpair) dpair[t] = split_pair(d);
    if (dscale) dscale[t] = sizeof(T) == 8 ? (T)(1.0 / d) : (T)(1.0 / sqrt(d));
  }
}

// offv_t[l][k] = offv[l][k] / sqrt(S_vv S_ww) in FP32 (unit-diagonal scaling)
__global__ void scaled_offdiag_kernel(DevGraph g, int32_t L, const double* __restrict__ offv,
                                      const float* __restrict__ dscale, float* __restrict__ offv_t) {
  const int64_t total = (int64_t)L * g.nv;
  const int64_t nadj = 2 * (int64_t)g.ne;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = t / g.nv;
    const int32_t v = (int32_t)(t - l * g.nv);
    const double sv = (double)dscale[t];
    for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
      const double sw = (double)dscale[l * g.nv + g.adj_nbr[k]];
      offv_t[l * nadj + k] = (float)(offv[l * nadj + k] * sv * sw);
    }
  }
}

// Neumann-Neumann preconditioner of the vertex system (Sec. 3, Phase 4, the
// Neumann step): P = D_G^-1 (sum_e (S^(e))^-1) D_G^-1, D_G = diag(vertex
// degree), with the 2x2 block inverses (S^(e))^-1 = [[a, -b], [-b, a]] / det,
// a = saa_e, b = sab_e, det = (a - b)(a + b) = c^2 sinh^2(theta) > 0. For
// incidence k (v -> w over edge e):
//   unscaled:  pc_v = sum_e a / det / d_v^2,   pn_k = -b / det / (d_v d_w);
//   scaled (the same operator on D^-1/2 S D^-1/2): D^1/2 P D^1/2, i.e.
//              pc_v = D_v sum_e a / det / d_v^2,
//              pn_k = -sqrt(D_v D_w) b / det / (d_v d_w).
template <typename T>
__global__ void nn_coeff_kernel(DevGraph g, int32_t L, const double* __restrict__ saa,
                                const double* __restrict__ sab, const double* __restrict__ diag,
                                int scaled, T* __restrict__ pc, T* __restrict__ pn) {
  const int64_t total = (int64_t)L * g.nv;
  const int64_t nadj = 2 * (int64_t)g.ne;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = t / g.nv;
    const int32_t v = (int32_t)(t - l * g.nv);
    const double dv = (double)(g.vptr[v + 1] - g.vptr[v]);
    const double Dv = diag[t];
    double acc = 0.0;
    for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
      const int64_t i = l * g.ne + g.adj_edge[k];
      const double a = saa[i], b = sab[i];
      const double det = (a - b) * (a + b);
      acc += a / det;
      const int32_t w = g.adj_nbr[k];
      const double dw = (double)(g.vptr[w + 1] - g.vptr[w]);
      double c = -b / det / (dv * dw);
      if (scaled) c *= sqrt(Dv * diag[l * g.nv + w]);
      pn[l * nadj + k] = (T)c;
    }
    pc[t] = (T)(acc / (dv * dv) * (scaled ? Dv : 1.0));
  }
}

int grid_for(int64_t total, int threads) {
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > sm_count() * 32) blocks = sm_count() * 32;
  return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace

template <typename T>
int launch_schur(const DevGraph& g, const DevNodes& nd, double kappa2, double* saa, double* sab,
                 double* diag, double* offv, SweepParams<T>* prm, T* dscale, T* offv_t,
                 cudaStream_t st, bool consistent, float2* dpair, float2* opair) {
  edge_blocks_kernel<T><<<grid_for((int64_t)nd.L * g.ne, 256), 256, 0, st>>>(
      g, nd, kappa2, saa, sab, consistent ? nullptr : prm, consistent ? 1 : 0);
  vertex_diag_kernel<T><<<grid_for((int64_t)nd.L * g.nv, 256), 256, 0, st>>>(
      g, nd.L, saa, sab, diag, offv, dscale, dpair, opair);
  if constexpr (sizeof(T) == 4) {
    if (dscale && offv_t) {
      scaled_offdiag_kernel<<<grid_for((int64_t)nd.L * g.nv, 256), 256, 0, st>>>(g, nd.L, offv,
                                                                                 dscale, offv_t);
      return 3;
    }
  }
  return 2;
}
template <typename T>
void launch_nn_coeffs(const DevGraph& g, int32_t L, const double* saa, const double* sab,
                      const double* diag, bool scaled, T* pc, T* pn, cudaStream_t st) {
  nn_coeff_kernel<T><<<grid_for((int64_t)L * g.nv, 256), 256, 0, st>>>(g, L, saa, sab, diag,
                                                                      scaled ? 1 : 0, pc, pn);
}
template void launch_nn_coeffs<float>(const DevGraph&, int32_t, const double*, const double*,
                                      const double*, bool, float*, float*, cudaStream_t);
template void launch_nn_coeffs<double>(const DevGraph&, int32_t, const double*, const double*,
                                       const double*, bool, double*, double*, cudaStream_t);

template int launch_schur<float>(const DevGraph&, const DevNodes&, double, double*, double*,
                                 double*, double*, SweepParams<float>*, float*, float*,
                                 cudaStream_t, bool, float2*, float2*);
template int launch_schur<double>(const DevGraph&, const DevNodes&, double, double*, double*,
                                  double*, double*, SweepParams<double>*, double*, double*,
                                  cudaStream_t, bool, float2*, float2*);

}  // namespace grf
