// White noise of the consistent-mass comparison system (Eq. wh_def with the
// consistent mass of Sec. 3 Phase 2): W = R xi, M = R R^T the Cholesky factor
// with the DOFs in the order of the Phase 2 partition, the interior nodes edge
// by edge and then the vertices by kept id. In that order
//   R = [[R_II, 0], [X, R_S]],  X = M_GI R_II^-T,  R_S R_S^T = S_M,
// S_M = M_GG - M_GI M_II^-1 M_IG the vertex Schur complement of the mass.
// R_II is block diagonal: on an edge (h = h_e) M_II = tridiag(h/6, 2h/3, h/6)
// has the bidiagonal factor with pivots p_1 = 2h/3, p_{i+1} = 2h/3 - (h/6)^2 / p_i
// (R_ii = sqrt(p_i), R_{i+1,i} = (h/6) / R_ii), which reach their fixed point
// h (1/3 + sqrt(3)/6) to FP32 precision within a few steps. Hence per edge and
// sample: W_I = R_II xi_I (one forward pass) and the two entries of
// z = R_II^-T xi_I next to the end vertices (one backward pass), and per vertex
// W_v = sum over its edges (h/6) z_adj + (R_S xi_G)_v. R_S comes from the host
// (a sparse factorisation of S_M, once per graph); the per-sample work here is
// O(N) and runs in FP32 like the lumped noise of the mixed path.
#include "grf_internal.h"

namespace grf {
namespace {

constexpr int kPiv = 24;  // pivots kept before the fixed point

// On entry b holds the standard normals xi [n][S]; the interior rows become
// W_I, wv [nv][S] (zeroed) receives the vertices' X xi_I terms.
__global__ void cons_noise_edges_kernel(DevGraph g, int64_t S, float* __restrict__ b,
                                        float* __restrict__ wv) {
  const int64_t total = (int64_t)g.ne * S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = (int32_t)(t / S);
    const int64_t s = t - (int64_t)e * S;
    const int32_t m = g.nel[e] - 1;
    if (m <= 0) continue;
    const float h = (float)g.he[e];
    const float a = h * (1.f / 6.f), d = h * (2.f / 3.f);
    float lp[kPiv];
    float p = d;
#pragma unroll
    for (int i = 0; i < kPiv; ++i) {
      lp[i] = sqrtf(p);
      p = d - a * a / p;
    }
    const float lstar = sqrtf(h * (1.f / 3.f + 0.28867513459481287f));  // sqrt(3)/6
    float* col = b + ((int64_t)g.nv + g.ioff[e]) * S + s;
    // z = R_II^-T xi_I from the far end: z_i = (xi_i - (a / l_i) z_{i+1}) / l_i
    const float lm = m - 1 < kPiv ? lp[m - 1] : lstar;
    const float zm = col[(int64_t)(m - 1) * S] / lm;
    float z = zm;
    for (int32_t i = m - 2; i >= 0; --i) {
      const float li = i < kPiv ? lp[i] : lstar;
      z = (col[(int64_t)i * S] - (a / li) * z) / li;
    }
    // W_I = R_II xi_I in place: W_i = l_i xi_i + (a / l_{i-1}) xi_{i-1}
    float prev = 0.f, lprev = 1.f;
    for (int32_t i = 0; i < m; ++i) {
      const float li = i < kPiv ? lp[i] : lstar;
      const float xi = col[(int64_t)i * S];
      col[(int64_t)i * S] = li * xi + (i > 0 ? (a / lprev) * prev : 0.f);
      prev = xi;
      lprev = li;
    }
    atomicAdd(wv + (int64_t)g.eu[e] * S + s, a * z);   // node 1 is next to edge_u
    atomicAdd(wv + (int64_t)g.ev[e] * S + s, a * zm);  // node m is next to edge_v
  }
}

// wv[v][s] += (R_S xi_G)_v: row v of the lower factor (CSR) against the
// vertices' normals, still in b's vertex rows.
__global__ void cons_noise_vertices_kernel(DevGraph g, int64_t S, const int64_t* __restrict__ rp,
                                           const int32_t* __restrict__ rc,
                                           const float* __restrict__ rv,
                                           const float* __restrict__ b, float* __restrict__ wv) {
  const int64_t total = (int64_t)g.nv * S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / S, s = t - v * S;
    float acc = 0.f;
    for (int64_t k = rp[v]; k < rp[v + 1]; ++k) acc = fmaf(rv[k], b[(int64_t)rc[k] * S + s], acc);
    wv[t] += acc;
  }
}

__global__ void cons_noise_copy_kernel(int64_t count, const float* __restrict__ wv,
                                       float* __restrict__ b) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    b[t] = wv[t];
}

int blocks_for(int64_t total, int threads, int n_sm) {
  int64_t bl = (total + threads - 1) / threads;
  const int64_t cap = (int64_t)(n_sm > 0 ? n_sm : 1) * 16;
  if (bl > cap) bl = cap;
  return bl < 1 ? 1 : (int)bl;
}

__global__ void minor_to_major_kernel(int64_t n, int64_t S, const float* __restrict__ b,
                                      double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * S;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / n, j = t - s * n;
    out[t] = (double)b[j * S + s];
  }
}

}  // namespace

void launch_minor_to_major(int64_t n, int64_t S, const float* b, double* out, cudaStream_t st) {
  minor_to_major_kernel<<<blocks_for(n * S, 256, sm_count()), 256, 0, st>>>(n, S, b, out);
}

int launch_cons_noise(const DevGraph& g, int64_t S, float* b, float* wv, const int64_t* rp,
                      const int32_t* rc, const float* rv, int n_sm, cudaStream_t st) {
  const int64_t nvs = (int64_t)g.nv * S;
  cudaMemsetAsync(wv, 0, sizeof(float) * (size_t)nvs, st);
  cons_noise_edges_kernel<<<blocks_for((int64_t)g.ne * S, 256, n_sm), 256, 0, st>>>(g, S, b, wv);
  cons_noise_vertices_kernel<<<blocks_for(nvs, 256, n_sm), 256, 0, st>>>(g, S, rp, rc, rv, b, wv);
  cons_noise_copy_kernel<<<blocks_for(nvs, 256, n_sm), 256, 0, st>>>(nvs, wv, b);
  return 3;
}

}  // namespace grf
