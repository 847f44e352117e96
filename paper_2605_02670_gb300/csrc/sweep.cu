// Node-parallel interior sweeps for FP32 interiors (Sec. 3, Phases 3 and 5).
//
// One warp per (edge, group of 4 samples). Lane j owns the quadrature nodes
// l = j + 32 n (n < NL) and runs their tridiagonal eliminations along the edge
// one interior node at a time, for the four samples at once. All lanes read the
// same noise row at the same step, so one row load feeds 4 x NL eliminations
// per direction, and nothing crosses lanes except the sum over nodes.
//
// With 2 + delta = 2 cosh(theta), T = tridiag(-1, 2 + delta, -1) has the
// elimination pivots p_j = 1 + q_j from either end, q_1 = 1 + delta,
// q_{j+1} = delta + q_j / (1 + q_j), in closed form
//   q_j = delta / 2 + sinh(theta) coth(j theta),
// which equals q* = delta / 2 + sinh(theta) in FP32 once j theta >= 9; from
// there on the sweeps run with the constant pivot 1 + q*.
//
// condense: the end values of T^{-1} b_I (Eq. local_reduced_schur), one
//   elimination from each end, as in thomas.cu.
// recover: U_K = sum_l x_K^(l), T_l x^(l) = sc_l b + x_a e_1 + x_b e_m
//   (Eq. internal_recovery, weights folded into sc_l and x_a, x_b), by the
//   twisted factorisation of T at every node K:
//     x_K = (y_K + z_K - r_K) / gamma_K,   gamma_K = q_K + q'_K - delta,
//   y the elimination from node 1 (pivots 1 + q_K), z the elimination from
//   node m (pivots 1 + q'_K, q'_K = q_{m+1-K}), r the right-hand side. With
//   z_K - r_K = z_{K+1} / (1 + q'_{K+1}) there is no cancellation. Pass A runs
//   from node 1 and writes sum_l sc_l y_K / gamma_K into the output, pass B
//   runs from node m and adds sum_l sc_l (z_K - r_K) / gamma_K: two sweeps,
//   no back substitution and nothing stored per node l. gamma_K needs the
//   pivot excess of the other direction, q* away from that end and the closed
//   form near it. The sweeps run on b + (x_a / sc_l) e_1 + (x_b / sc_l) e_m;
//   the factor sc_l is applied with 1 / gamma_K.
//
// The sum over nodes at a node K: FP32 over a lane's NL nodes, then an FP32
// butterfly over the 32 lanes (a pairwise tree).
#include <cuda_runtime.h>

#include "grf_internal.h"

namespace grf {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 4;  // units (warps) per CTA
constexpr int kS = 4;      // samples per unit
// resident CTAs per SM the register budget aims at (128 or 168 registers, no spills)
constexpr int min_blocks(int nl) { return nl <= 5 ? 4 : 3; }
constexpr float kConvTheta = 9.0f;

__device__ __forceinline__ float rcpf(float x) { return __fdividef(1.0f, x); }

// Per (unit, node) constants of one lane slot.
struct NodeK {
  float dl, sc, sh, th;  // delta, sc = w_l / c_l, sinh(theta), theta
  float qs, rps, cs;     // q*, 1 / (1 + q*), sc / (2 sinh(theta))
  int kc;                // q_j = q* for j >= kc
};

// 1 - exp(-a) for a >= 0 without cancellation (series below 0.25, truncation
// < 5e-8 relative)
__device__ __forceinline__ float one_minus_exp(float a) {
  const float ser =
      a * (1.f - a * (0.5f - a * (1.f / 6 - a * (1.f / 24 - a * (1.f / 120 - a * (1.f / 720))))));
  return a < 0.25f ? ser : 1.0f - __expf(-a);
}

__device__ __forceinline__ NodeK node_consts(const SweepParams<float>& p, int m, bool live) {
  NodeK k;
  if (!live) {  // an empty slot: contributes nothing
    k.dl = 1.f; k.sc = 0.f; k.sh = 1.f; k.th = 1.f;
  } else {
    k.dl = p.delta; k.sc = p.sc; k.sh = p.sh; k.th = p.theta;
  }
  k.qs = 0.5f * k.dl + k.sh;
  k.rps = rcpf(1.0f + k.qs);
  k.cs = k.sc * rcpf(2.0f * k.sh);
  const float kcf = ceilf(kConvTheta / k.th);
  k.kc = kcf < (float)(m + 1) ? (kcf < 2.f ? 2 : (int)kcf) : m + 1;
  return k;
}

// Row `row` of the unit's 4 samples (vec: S % 4 == 0, 16-byte aligned); zeros
// when !ok.
__device__ __forceinline__ float4 fetch_row(const float* rows, int64_t S, int row, bool vec,
                                            int kv, bool ok) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!ok) return v;
  const float* p = rows + (int64_t)row * S;
  if (vec) return __ldg(reinterpret_cast<const float4*>(p));
  v.x = __ldg(p);
  if (kv > 1) v.y = __ldg(p + 1);
  if (kv > 2) v.z = __ldg(p + 2);
  if (kv > 3) v.w = __ldg(p + 3);
  return v;
}

// Steps j = j0..j1 of a sweep read row ri(j). They run in chunks of 32: the
// chunk's rows sit in this warp's shared buffer (one row per lane, written
// from the prefetch register), and each lane already holds its row of the next
// chunk in flight while the current one is swept.
template <typename RowOf, typename Step>
__device__ __forceinline__ void chunked_sweep(float4* buf, int lane, const float* rows, int64_t S,
                                              bool vec, int kv, int32_t j0, int32_t j1, RowOf ri,
                                              Step step) {
  if (j0 > j1) return;
  float4 pf = fetch_row(rows, S, ri(j0 + lane), vec, kv, j0 + lane <= j1);
  for (int32_t c0 = j0; c0 <= j1; c0 += 32) {
    __syncwarp();
    buf[lane] = pf;
    __syncwarp();
    const int32_t jn = c0 + 32 + lane;
    pf = fetch_row(rows, S, ri(jn), vec, kv, jn <= j1);
    const int32_t cnt = min(32, j1 - c0 + 1);
#pragma unroll 1
    for (int32_t i = 0; i < cnt; ++i) step(c0 + i, buf[i]);
  }
}

// Sum of c[0..3] over the warp for sample lane >> 3: reduce-scatter, 6 shuffles.
__device__ __forceinline__ float warp_sum4(const float (&c)[kS], int lane) {
  const bool hi = lane >= 16;
  float k0 = hi ? c[2] : c[0], k1 = hi ? c[3] : c[1];
  const float s0 = hi ? c[0] : c[2], s1 = hi ? c[1] : c[3];
  k0 += __shfl_xor_sync(kFull, s0, 16);
  k1 += __shfl_xor_sync(kFull, s1, 16);
  const bool odd = lane & 8;
  float v = odd ? k1 : k0;
  v += __shfl_xor_sync(kFull, odd ? k0 : k1, 8);
  v += __shfl_xor_sync(kFull, v, 4);
  v += __shfl_xor_sync(kFull, v, 2);
  v += __shfl_xor_sync(kFull, v, 1);
  return v;
}

struct Unit {
  bool live;
  int32_t e, m, va, vb;
  int64_t s0, off;
  int kv;
};

__device__ __forceinline__ Unit unit_of(const DevGraph& g, const int32_t* edges, int64_t nsg,
                                        int64_t u, int64_t n_units, int64_t S) {
  Unit t;
  t.live = u < n_units;
  t.e = t.live ? (edges ? edges[u / nsg] : (int32_t)(u / nsg)) : 0;
  t.s0 = t.live ? (u % nsg) * kS : 0;
  t.m = t.live ? g.nel[t.e] - 1 : 0;
  t.off = t.live ? g.ioff[t.e] : 0;
  t.va = t.live ? g.eu[t.e] : 0;
  t.vb = t.live ? g.ev[t.e] : 0;
  t.kv = (int)(S - t.s0 < kS ? S - t.s0 : kS);
  return t;
}

// ---- condensation: both end eliminations in one pass
// Step j carries the elimination into node j from node j - 1 (pivot 1 + q_{j-1}),
// from node 1 forward (y) and from node m backward (z, rows m - j).
template <int NL>
__global__ void __launch_bounds__(32 * kWarps, min_blocks(NL))
    condense_nodes_kernel(DevGraph g, int32_t L, int64_t S, const float* __restrict__ b,
                          const SweepParams<float>* __restrict__ prm,
                          const int32_t* __restrict__ edges, int32_t n_edges,
                          double* __restrict__ gvec) {
  __shared__ float4 stage[kWarps][2][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nsg = (S + kS - 1) / kS;
  const int64_t n_units = (int64_t)n_edges * nsg;
  const bool vec = (S % kS) == 0;
  for (int64_t u = (int64_t)blockIdx.x * kWarps + wid; u < n_units;
       u += (int64_t)gridDim.x * kWarps) {
    const Unit t = unit_of(g, edges, nsg, u, n_units, S);
    const int32_t m = t.m;
    if (m <= 0) continue;  // uniform across the warp
    float dl[NL], rps[NL], q[NL], rp[NL];
    int kcw = 2;
#pragma unroll
    for (int n = 0; n < NL; ++n) {
      const int l = lane + 32 * n;
      const bool on = l < L;
      const NodeK k = node_consts(on ? prm[(int64_t)l * g.ne + t.e] : SweepParams<float>{}, m, on);
      dl[n] = k.dl;
      rps[n] = k.rps;
      q[n] = 0.f;
      rp[n] = 0.f;
      kcw = max(kcw, k.kc);
    }
    kcw = __reduce_max_sync(kFull, kcw);
    const float* rows = b + (g.nv + t.off) * S + t.s0;
    float yf[NL][kS], yr[NL][kS];
#pragma unroll
    for (int n = 0; n < NL; ++n)
#pragma unroll
      for (int s = 0; s < kS; ++s) yf[n][s] = yr[n][s] = 0.f;
    // forward rows 0.. and backward rows m-1.. interleaved: two staged streams
    float4* bf = stage[wid][0];
    float4* br = stage[wid][1];
    float4 pff = fetch_row(rows, S, lane, vec, t.kv, lane < m);
    float4 pfr = fetch_row(rows, S, m - 1 - lane, vec, t.kv, lane < m);
    for (int32_t c0 = 1; c0 <= m; c0 += 32) {
      __syncwarp();
      bf[lane] = pff;
      br[lane] = pfr;
      __syncwarp();
      const int32_t jn = c0 + 32 + lane;  // next chunk's node for this lane
      pff = fetch_row(rows, S, jn - 1, vec, t.kv, jn <= m);
      pfr = fetch_row(rows, S, m - jn, vec, t.kv, jn <= m);
      const int32_t cnt = min(32, m - c0 + 1);
      if (c0 > kcw) {  // every pivot at the fixed point
        for (int32_t i = 0; i < cnt; ++i) {
          const float4 f = bf[i], r = br[i];
          const float fv[kS] = {f.x, f.y, f.z, f.w}, rv[kS] = {r.x, r.y, r.z, r.w};
#pragma unroll
          for (int n = 0; n < NL; ++n)
#pragma unroll
            for (int s = 0; s < kS; ++s) {
              yf[n][s] = fmaf(rps[n], yf[n][s], fv[s]);
              yr[n][s] = fmaf(rps[n], yr[n][s], rv[s]);
            }
        }
      } else {  // the recurrence runs on past convergence: its fixed point attracts
        for (int32_t i = 0; i < cnt; ++i) {
          const int32_t j = c0 + i;
          const float4 f = bf[i], r = br[i];
          const float fv[kS] = {f.x, f.y, f.z, f.w}, rv[kS] = {r.x, r.y, r.z, r.w};
#pragma unroll
          for (int n = 0; n < NL; ++n) {
#pragma unroll
            for (int s = 0; s < kS; ++s) {
              yf[n][s] = fmaf(rp[n], yf[n][s], fv[s]);  // rp = 0 at j = 1
              yr[n][s] = fmaf(rp[n], yr[n][s], rv[s]);
            }
            // pivot of node j for the next step
            q[n] = j == 1 ? 1.0f + dl[n] : fmaf(q[n], rp[n], dl[n]);
            rp[n] = rcpf(1.0f + q[n]);
          }
        }
      }
    }
    // end values: (T^{-1} b)_m = y_m / p_m next to edge_v, (T^{-1} b)_1 next to edge_u
#pragma unroll
    for (int n = 0; n < NL; ++n) {
      const int l = lane + 32 * n;
      if (l >= L) continue;
      const float rpm = m > kcw ? rps[n] : rp[n];
      double* gl = gvec + (int64_t)l * S * g.nv;
#pragma unroll
      for (int s = 0; s < kS; ++s) {
        if (s < t.kv) {
          atomicAdd(gl + (t.s0 + s) * g.nv + t.vb, (double)(yf[n][s] * rpm));
          atomicAdd(gl + (t.s0 + s) * g.nv + t.va, (double)(yr[n][s] * rpm));
        }
      }
    }
  }
}

// ---- recovery: two passes of the twisted factorisation
//
// Pass kB = false runs from node 1 (j = K), kB = true from node m (j = m + 1 - K).
// 1 / gamma_K is the diagonal of T^{-1} in closed form,
//   1 / gamma = F(j) F(m + 1 - j) / (2 sinh(theta) F(m + 1)),  F(i) = 1 - exp(-2 i theta),
// so the factor of a node is sc / (2 sinh(theta)) times F of the distances to
// both ends. Regions: the two boundary nodes (x_a, x_b enter there), near the
// start (j <= kcw: own pivots by the recurrence, F(j) by F(j+1) = F(j) +
// exp(-2 j theta) F(1)), the middle (both pivots at the fixed point, constant
// factor), near the other end (j > m + 1 - kcw: F(m + 1 - j) from exp,
// re-anchored every 8 nodes and at the last 8). Edges shorter than 2 kcw take
// the near kind of step throughout, with F of the far end from the same
// anchored exp products as the far region.
// Each region loads the constants it needs, so few stay live across regions.
// Results go to out at node K for sample s in lane 8 s + ((K - 1) & 7), stored
// in aligned blocks of 8 nodes; pass B reads back what the same lane wrote in
// pass A and adds to it.
template <int NL, bool kB, typename OutT>
__device__ __forceinline__ void twisted_pass(const Unit& t, int lane, int64_t S, int64_t n_dofs,
                                             int32_t nv, int32_t L, const float* rows, bool vec,
                                             const SweepParams<float>* pe, int64_t pstride,
                                             const float* xs, const float* xe, int64_t xstride,
                                             int kcw, float4* buf, OutT* out) {
  const int32_t m = t.m;
  const int sl = lane >> 3;  // this lane's sample in the sums
  const bool store_lane = t.live && sl < t.kv;
  OutT* orow = out + (t.s0 + (sl < t.kv ? sl : 0)) * n_dofs + nv + t.off;  // + K - 1
  auto prm_of = [&](int n) {
    const int l = lane + 32 * n;
    SweepParams<float> p;
    if (l < L) {
      p = pe[(int64_t)l * pstride];
    } else {  // an empty slot: contributes nothing
      p.delta = 1.f; p.sc = 0.f; p.sh = 1.f; p.theta = 1.f;
    }
    return p;
  };
  float y[NL][kS], rp[NL];
#pragma unroll
  for (int n = 0; n < NL; ++n) {
    rp[n] = 0.f;
#pragma unroll
    for (int s = 0; s < kS; ++s) y[n][s] = 0.f;
  }
  float keep = 0.f;  // this lane's node of the current block of 8
  auto finish = [&](int j, float (&c)[kS]) {
    const float v = warp_sum4(c, lane);
    const int K = kB ? m + 1 - j : j;
    if ((lane & 7) == ((K - 1) & 7)) keep = v;
    // flush the block of 8 nodes that ends here (K = 0 mod 8 or m going up,
    // K = 1 mod 8 going down)
    const bool end = kB ? ((K - 1) & 7) == 0 : ((K & 7) == 0 || K == m);
    if (end) {
      const int Kl = ((K - 1) & ~7) + (lane & 7);  // 0-based node of this lane
      if (store_lane && Kl < m) {
        if (kB)
          orow[Kl] = (OutT)((double)orow[Kl] + (double)keep);
        else
          orow[Kl] = (OutT)keep;
      }
    }
  };
  auto row_of = [&](int j) { return kB ? m - j : j - 1; };
  const bool overlap = m + 1 < 2 * kcw;
  // a boundary node (j = 1 or j = m): the factor from its closed form; the
  // carry rp[] holds 1 / p_{j-1} and on return 1 / p_1
  auto edge_step = [&](int j, float4 r4) {
    const float r[kS] = {r4.x, r4.y, r4.z, r4.w};
    float c[kS] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int n = 0; n < NL; ++n) {
      const SweepParams<float> p = prm_of(n);
      const int l = lane + 32 * n;
      const float isc = p.sc != 0.f ? rcpf(p.sc) : 0.f;
      float add[kS] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int s = 0; s < kS; ++s) {
        if (p.sc != 0.f && s < t.kv) {
          if (j == 1) add[s] += xs[(int64_t)l * xstride + s] * isc;
          if (j == m) add[s] += xe[(int64_t)l * xstride + s] * isc;
        }
      }
      const float two = 2.0f * p.theta;
      const float g = p.sc * rcpf(2.0f * p.sh) * one_minus_exp(two * (float)j) *
                      one_minus_exp(two * (float)(m + 1 - j)) *
                      rcpf(one_minus_exp(two * (float)(m + 1)));
#pragma unroll
      for (int s = 0; s < kS; ++s) {
        const float tc = rp[n] * y[n][s];
        y[n][s] = r[s] + add[s] + tc;
        c[s] = fmaf(g, kB ? tc : y[n][s], c[s]);
      }
      // 1 / p_1 for the carry into node 2 (q_1 = 1 + delta); after node m no carry
      rp[n] = rcpf(2.0f + p.delta);
      asm volatile("" ::: "memory");  // one slot's loads at a time: fewer live registers
    }
    finish(j, c);
  };
  chunked_sweep(buf, lane, rows, S, vec, t.kv, 1, 1, row_of, edge_step);
  if (m == 1) return;
  // near region j = 2 .. e1. The pivot recurrence runs on past the nodes whose
  // pivot has converged: the fixed point is attracting, so it stays there.
  const int e1 = overlap ? m - 1 : min(kcw, m - 1);
  {
    // gf = sc F(j) / (2 sinh(theta)) and its increment w = sc F(1) exp(-2 j theta) / (2 sinh(theta))
    float q[NL], gf[NL], w[NL], ed[NL], dl[NL], thn[NL], nrm[NL], ef[NL], e2[NL];
#pragma unroll
    for (int n = 0; n < NL; ++n) {
      const SweepParams<float> p = prm_of(n);
      dl[n] = p.delta;
      const float cs = p.sc * rcpf(2.0f * p.sh);
      const float d1 = one_minus_exp(2.0f * p.theta);  // F(1)
      ed[n] = 1.0f - d1;                               // exp(-2 theta)
      // state at j = 2: q_2, F(2), exp(-4 theta)
      const float q1 = 1.0f + p.delta;
      q[n] = fmaf(q1, rp[n], p.delta);
      gf[n] = cs * fmaf(ed[n], d1, d1);
      w[n] = cs * d1 * ed[n] * ed[n];
      thn[n] = p.theta;
      nrm[n] = overlap ? rcpf(one_minus_exp(2.0f * (float)(m + 1) * p.theta)) : 1.0f;
      ef[n] = 0.f;  // exp(-2 (m + 1 - j) theta), anchored at the first step
      e2[n] = __expf(fminf(2.0f * p.theta, 80.0f));
    }
    chunked_sweep(buf, lane, rows, S, vec, t.kv, 2, e1, row_of, [&](int j, float4 r4) {
      const float r[kS] = {r4.x, r4.y, r4.z, r4.w};
      float c[kS] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int n = 0; n < NL; ++n) {
        float gsc = gf[n];
        if (overlap) {  // uniform: the far factor F(m + 1 - j) / F(m + 1)
          const int jf = m + 1 - j;
          float ff;
          if ((jf & 7) == 0 || jf <= 8 || j == 2) {  // re-anchor
            const float a = 2.0f * (float)jf * thn[n];
            ef[n] = __expf(-a);
            ff = one_minus_exp(a);
          } else {
            ef[n] *= e2[n];
            ff = 1.0f - ef[n];
          }
          gsc *= ff * nrm[n];
        }
        if (kB) {
          const float gr = gsc * rp[n];
#pragma unroll
          for (int s = 0; s < kS; ++s) {
            c[s] = fmaf(gr, y[n][s], c[s]);
            y[n][s] = fmaf(rp[n], y[n][s], r[s]);
          }
        } else {
#pragma unroll
          for (int s = 0; s < kS; ++s) {
            y[n][s] = fmaf(rp[n], y[n][s], r[s]);
            c[s] = fmaf(gsc, y[n][s], c[s]);
          }
        }
        // pivot of node j for the carry into j + 1, then q_{j+1}, F(j+1)
        rp[n] = rcpf(1.0f + q[n]);
        q[n] = fmaf(q[n], rp[n], dl[n]);
        gf[n] += w[n];
        w[n] *= ed[n];
      }
      finish(j, c);
    });
  }
  // middle: both pivots at the fixed point, constant factor
  const int s3 = overlap ? m : max(m + 2 - kcw, e1 + 1);  // first far step
  if (s3 - 1 >= e1 + 1) {
    float rps[NL], cf[NL];
#pragma unroll
    for (int n = 0; n < NL; ++n) {
      const SweepParams<float> p = prm_of(n);
      rps[n] = rcpf(1.0f + 0.5f * p.delta + p.sh);
      const float cs = p.sc * rcpf(2.0f * p.sh);
      cf[n] = kB ? cs * rps[n] : cs;
      rp[n] = rps[n];
    }
    chunked_sweep(buf, lane, rows, S, vec, t.kv, e1 + 1, s3 - 1, row_of, [&](int j, float4 r4) {
      const float r[kS] = {r4.x, r4.y, r4.z, r4.w};
      float c[kS] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int n = 0; n < NL; ++n) {
#pragma unroll
        for (int s = 0; s < kS; ++s) {
          if (kB) {  // the carried part rps z_{j-1} enters the sum
            c[s] = fmaf(cf[n], y[n][s], c[s]);
            y[n][s] = fmaf(rps[n], y[n][s], r[s]);
          } else {
            y[n][s] = fmaf(rps[n], y[n][s], r[s]);
            c[s] = fmaf(cf[n], y[n][s], c[s]);
          }
        }
      }
      finish(j, c);
    });
  }
  // far region j = s3 .. m - 1: own pivot at the fixed point, F(m + 1 - j) from exp
  if (!overlap && s3 <= m - 1) {
    float rps[NL], cs[NL], thn[NL], e2[NL], ef[NL];
#pragma unroll
    for (int n = 0; n < NL; ++n) {
      const SweepParams<float> p = prm_of(n);
      rps[n] = rcpf(1.0f + 0.5f * p.delta + p.sh);
      cs[n] = p.sc * rcpf(2.0f * p.sh);
      thn[n] = p.theta;
      // exp(2 theta), capped: where it would overflow, exp(-2 jf theta) is 0 already
      e2[n] = __expf(fminf(2.0f * p.theta, 80.0f));
      ef[n] = 0.f;
      rp[n] = rps[n];
    }
    chunked_sweep(buf, lane, rows, S, vec, t.kv, s3, m - 1, row_of, [&](int j, float4 r4) {
      const float r[kS] = {r4.x, r4.y, r4.z, r4.w};
      float c[kS] = {0.f, 0.f, 0.f, 0.f};
      const int jf = m + 1 - j;
      const bool anchor = (jf & 7) == 0 || jf <= 8 || j == s3;
#pragma unroll
      for (int n = 0; n < NL; ++n) {
        float ff;
        if (anchor) {  // uniform branch
          const float a = 2.0f * (float)jf * thn[n];
          ef[n] = __expf(-a);
          ff = one_minus_exp(a);
        } else {
          ef[n] *= e2[n];
          ff = 1.0f - ef[n];
        }
        const float gsc = cs[n] * ff;
        if (kB) {
          const float gr = gsc * rps[n];
#pragma unroll
          for (int s = 0; s < kS; ++s) {
            c[s] = fmaf(gr, y[n][s], c[s]);
            y[n][s] = fmaf(rps[n], y[n][s], r[s]);
          }
        } else {
#pragma unroll
          for (int s = 0; s < kS; ++s) {
            y[n][s] = fmaf(rps[n], y[n][s], r[s]);
            c[s] = fmaf(gsc, y[n][s], c[s]);
          }
        }
      }
      finish(j, c);
    });
  }
  chunked_sweep(buf, lane, rows, S, vec, t.kv, m, m, row_of, edge_step);
}

template <int NL, typename OutT>
__global__ void __launch_bounds__(32 * kWarps, min_blocks(NL))
    recover_nodes_kernel(DevGraph g, int32_t L, int64_t S, const float* __restrict__ b,
                         const SweepParams<float>* __restrict__ prm,
                         const float* __restrict__ xw, const int32_t* __restrict__ edges,
                         int32_t n_edges, OutT* __restrict__ out) {
  __shared__ float4 stage[kWarps][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nsg = (S + kS - 1) / kS;
  const int64_t n_units = (int64_t)n_edges * nsg;
  const bool vec = (S % kS) == 0;
  for (int64_t u = (int64_t)blockIdx.x * kWarps + wid; u < n_units;
       u += (int64_t)gridDim.x * kWarps) {
    const Unit t = unit_of(g, edges, nsg, u, n_units, S);
    if (t.m <= 0) continue;  // uniform across the warp
    const SweepParams<float>* pe = prm + t.e;
    int kcw = 2;
#pragma unroll
    for (int n = 0; n < NL; ++n) {
      const int l = lane + 32 * n;
      if (l < L) {
        const float kcf = ceilf(kConvTheta / pe[(int64_t)l * g.ne].theta);
        const int kc = kcf < (float)(t.m + 1) ? (kcf < 2.f ? 2 : (int)kcf) : t.m + 1;
        kcw = max(kcw, kc);
      }
    }
    kcw = __reduce_max_sync(kFull, kcw);
    const float* rows = b + (g.nv + t.off) * S + t.s0;
    // x_a, x_b of node l = w_l u^(l) at the edge's ends: xw[l][v][s]
    const int64_t xstride = (int64_t)g.nv * S;
    const float* xa = xw + (int64_t)t.va * S + t.s0;
    const float* xb = xw + (int64_t)t.vb * S + t.s0;
    twisted_pass<NL, false, OutT>(t, lane, S, g.n, g.nv, L, rows, vec, pe, g.ne, xa, xb, xstride,
                                  kcw, stage[wid], out);
    twisted_pass<NL, true, OutT>(t, lane, S, g.n, g.nv, L, rows, vec, pe, g.ne, xb, xa, xstride,
                                 kcw, stage[wid], out);
  }
}

int grid_units(int64_t units) {
  int64_t blocks = (units + kWarps - 1) / kWarps;
  if (blocks > sm_count() * 16) blocks = sm_count() * 16;
  return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace

int node_sweep_slots(int32_t L) { return (L + 31) / 32; }

bool node_sweep_fits(int32_t L) { return L >= 1 && node_sweep_slots(L) <= kNodeSweepMaxNL; }

int launch_condense_nodes(const DevGraph& g, int32_t L, int64_t S, const float* b,
                          const SweepParams<float>* prm, const int32_t* edges, int32_t n_edges,
                          double* gvec, cudaStream_t st) {
  if (n_edges <= 0) return 0;
  const int64_t units = (int64_t)n_edges * ((S + kS - 1) / kS);
  const int blocks = grid_units(units);
#define GRF_C(NL)                                                                            \
  condense_nodes_kernel<NL><<<blocks, 32 * kWarps, 0, st>>>(g, L, S, b, prm, edges, n_edges, \
                                                           gvec)
  switch (node_sweep_slots(L)) {
    case 1: GRF_C(1); break;
    case 2: GRF_C(2); break;
    case 3: GRF_C(3); break;
    case 4: GRF_C(4); break;
    case 5: GRF_C(5); break;
    case 6: GRF_C(6); break;
    case 7: GRF_C(7); break;
    default: GRF_C(8); break;
  }
#undef GRF_C
  return 1;
}

template <typename OutT>
int launch_recover_nodes(const DevGraph& g, int32_t L, int64_t S, const float* b,
                         const SweepParams<float>* prm, const float* xw, const int32_t* edges,
                         int32_t n_edges, OutT* out, cudaStream_t st) {
  if (n_edges <= 0) return 0;
  const int64_t units = (int64_t)n_edges * ((S + kS - 1) / kS);
  const int blocks = grid_units(units);
#define GRF_R(NL)                                                                  \
  recover_nodes_kernel<NL, OutT><<<blocks, 32 * kWarps, 0, st>>>(g, L, S, b, prm, xw, \
                                                                 edges, n_edges, out)
  switch (node_sweep_slots(L)) {
    case 1: GRF_R(1); break;
    case 2: GRF_R(2); break;
    case 3: GRF_R(3); break;
    case 4: GRF_R(4); break;
    case 5: GRF_R(5); break;
    case 6: GRF_R(6); break;
    case 7: GRF_R(7); break;
    default: GRF_R(8); break;
  }
#undef GRF_R
  return 1;
}

template int launch_recover_nodes<float>(const DevGraph&, int32_t, int64_t, const float*,
                                         const SweepParams<float>*, const float*, const int32_t*,
                                         int32_t, float*, cudaStream_t);
template int launch_recover_nodes<double>(const DevGraph&, int32_t, int64_t, const float*,
                                          const SweepParams<float>*, const float*,
                                          const int32_t*, int32_t, double*, cudaStream_t);

}  // namespace grf
