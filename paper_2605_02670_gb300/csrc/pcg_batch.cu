// Jacobi-PCG on the vertex Schur systems S^(l) u = g (Eq. global_schur; Sec. 3,
// Phase 4) for graphs whose vectors do not fit on chip: one CTA per (node l,
// group of 8 samples), the group's vectors stored as rows of 8 samples per
// vertex ([V][8], one 32-byte sector), so that every load of the node's matrix
// (incidence list, scaled block) serves the 8 samples and every vector access
// is a whole sector.
//
// Mixed precision: FP32 CG on the Jacobi-scaled system (D^-1/2 S D^-1/2) e =
// D^-1/2 r inside iterative refinement on S x~ = g~, g~ = g / ||g||. The
// refinement keeps its iterate x~ and right-hand side g~ as FP32 pairs
// (hi + lo, 48 significant bits), reads the FP64 blocks as pairs too, and
// forms r~ = g~ - S x~ as a compensated dot product (each product split exactly
// by an FMA, each sum by TwoSum; Ogita, Rump and Oishi's Dot2), accurate to a
// few units of 2^-48 of its terms, so no FP64 instruction runs in the
// refinement loop: FP64 issues at a small fraction of the FP32 rate. FP64
// remains in the norms of g, its split into pairs, the per-sample decisions
// and the final x = ||g|| (x~hi + x~lo).
// The dot products are FP32 partial sums over at most 16 vertices per thread,
// accumulated as FP32 pairs and summed in FP64 across the CTA; the CG scalars
// alpha, beta are FP64; the vector updates are FP32.
//
// A thread owns 4 of the group's samples (one 16-byte half row) of one vertex
// per step. The vertex's first four neighbours and its incidence-list start
// and degree come from one record per vertex, so every neighbour row and its
// coefficient are requested at once after a single dependent load (further
// neighbours, rare on these graphs, walk the incidence list).
// The per-sample CG state lives in shared memory; after each CTA reduction one
// thread per sample takes its decisions in FP64.
//
// One inner iteration is two passes over the vertices with one CTA reduction
// each, and moves 8 vector rows per vertex (instead of 10-11 for the textbook
// ordering):
//   pass A: p' = r + beta p (double-buffered: the neighbours' p' are formed
//           from their r and p, nothing is read that this pass writes),
//           q = S p' for the own vertex, partial p'.q;
//   pass B: q = S p' again (gathers of p', which stay in L1/L2), d += alpha p',
//           r -= alpha q, partial r.r.
// Every loop is bounded by max_iter; no CTA waits on another.
#include "grf_internal.h"

namespace grf {
namespace {

constexpr int kBT = 256;          // threads per CTA
constexpr int kSG = 8;            // samples per group: one 32-byte row per vertex
constexpr int kVP = kBT / 2;      // vertices per half-step (two threads per vertex row)
constexpr int kU = 1;             // vertices per thread per step
constexpr int kWarps = kBT / 32;
constexpr int kChunk = 16;        // FP32 partial sums over this many vertices
constexpr double kInnerRtol = 1e-5;
constexpr unsigned kFull = 0xffffffffu;

// Per-sample state of the group (one entry per sample, written by thread j).
struct SampleState {
  double rz, rz0, best, stop2, inner_e, rho, inv_g, gn;
  int32_t it, since;
  int32_t done, bad, cg, has_d, first;
  float af, bf;  // FP32 alpha, beta for the vector passes
  float scl;     // ||g|| / rho: r~ to the inner solve's right-hand side
  float xsc;     // rho / ||g||: the inner solution to the update of x~
};

struct BatchShared {
  double red[kWarps][kSG][2];
  SampleState st[kSG];
};

// (h, l) += t with h + l renormalised (two TwoSums): an FP32 pair.
__device__ __forceinline__ void ff_add(float& h, float& l, float t) {
  float s = __fadd_rn(h, t);
  float bv = __fsub_rn(s, h);
  float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bv)), __fsub_rn(t, bv));
  e = __fadd_rn(e, l);
  const float s2 = __fadd_rn(s, e);
  bv = __fsub_rn(s2, s);
  l = __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bv)), __fsub_rn(e, bv));
  h = s2;
}

// FP32 partial sums of 4 samples x N values, flushed every kChunk vertices
// into FP32 pairs (no FP64 instruction in the vertex loops).
template <int N>
struct Acc4 {
  float f[4][N], h[4][N], l[4][N];
  int c;
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < N; ++k) f[i][k] = h[i][k] = l[i][k] = 0.f;
    c = 0;
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < N; ++k) ff_add(h[i][k], l[i][k], f[i][k]), f[i][k] = 0.f;
  }
  __device__ __forceinline__ void tick() {
    if (++c == kChunk) flush(), c = 0;
  }
};

// Per-sample CTA sums: lanes of equal parity share a half row (4 samples).
// The warp sums run on the pairs; one FP64 value per (warp, sample) then goes
// through shared memory. After the call thread j < 8 holds the sums of sample
// j in out[k].
template <int N>
__device__ __forceinline__ void group_sum(Acc4<N>& a, BatchShared& sh, double (&out)[N]) {
  a.flush();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      float h = a.h[i][k], l = a.l[i][k];
#pragma unroll
      for (int o = 2; o < 32; o <<= 1) {
        const float oh = __shfl_xor_sync(kFull, h, o), ol = __shfl_xor_sync(kFull, l, o);
        ff_add(h, l, oh);
        l += ol;
      }
      if (lane < 2) sh.red[warp][4 * lane + i][k] = (double)h + (double)l;
    }
  __syncthreads();
  if (threadIdx.x < kSG) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double v = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) v += sh.red[w][threadIdx.x][k];
      out[k] = v;
    }
  }
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 fma4(float4 a, float4 x, float4 y) {  // a * x + y per lane
  return make_float4(fmaf(a.x, x.x, y.x), fmaf(a.y, x.y, y.y), fmaf(a.z, x.z, y.z),
                     fmaf(a.w, x.w, y.w));
}
__device__ __forceinline__ float4 fma1(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 sel4(const bool (&c)[4], float4 a, float4 b) {
  return make_float4(c[0] ? a.x : b.x, c[1] ? a.y : b.y, c[2] ? a.z : b.z, c[3] ? a.w : b.w);
}
__device__ __forceinline__ float get(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// (s, c) -= (ah + al)(xh + xl), s + c a running sum with its error term: the
// product ah xh = p + pe exactly (FMA), s - p = t + se exactly (TwoSum), the
// cross terms ah xl + al xh (and the dropped al xl, below 2^-46 of the
// product) need only FP32 accuracy. The _rn intrinsics keep the compiler from
// fusing the error-free steps.
__device__ __forceinline__ void ff_sub_prod(float& s, float& c, float ah, float al, float xh,
                                            float xl) {
  const float p = __fmul_rn(ah, xh);
  const float pe = __fmaf_rn(ah, xh, -p);
  const float mp = -p;
  const float t = __fadd_rn(s, mp);
  const float bv = __fsub_rn(t, s);
  const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(mp, bv));
  s = t;
  c += se - (pe + fmaf(ah, xl, al * xh));
}
// Bulk prefetch into L2 (TMA) of the vector rows of the vertices kPF steps
// ahead: the rows of a step are contiguous ([nv][8] floats), so one thread
// requests each vector's next block while the CTA works on the current one,
// and the step's own-row loads then hit L2 instead of waiting on DRAM.
constexpr int kPF = 4;
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void prefetch_rows(const float* rows, int32_t v0, int32_t nv) {
  const int32_t b = v0 + kPF * kVP;
  if (b >= nv) return;
  const int32_t n = nv - b < kVP ? nv - b : kVP;
  prefetch_l2(rows + (int64_t)b * kSG, (uint32_t)n * kSG * 4);
}
// The vertices' neighbour records of one step (vertices v0 + u kVP, u < kU):
// their first four neighbours and (incidence-list start, degree); past the
// end the records are empty.
__device__ __forceinline__ void load_ell(const int4* __restrict__ ell, int32_t v0, int32_t nv,
                                         int4 (&a)[kU], int2 (&b)[kU]) {
  const int2* __restrict__ info = reinterpret_cast<const int2*>(ell + nv);
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int32_t v = v0 + u * kVP;
    if (v < nv) {
      a[u] = __ldg(ell + v);
      b[u] = __ldg(info + v);
    } else {
      a[u] = make_int4(0, 0, 0, 0);
      b[u] = make_int2(0, 0);
    }
  }
}

}  // namespace

// gvec, xout: [L][S][nv] FP64 (right-hand sides in, solutions out); with
// g32 the right-hand sides come in FP32 in GH (same layout as the vectors) and
// gvec is not read.
// DP, OP: the FP64 blocks as FP32 pairs, [L][nv] and [L][2E].
// R, PA, PB, Dv, XH, XL, GH, GL: [L][ceil(S / 8)][nv][8] FP32 scratch.
__global__ void __launch_bounds__(kBT, 3) pcg_batch_kernel(
    DevGraph g, const int4* __restrict__ ell, int32_t L, int64_t S,
    const float2* __restrict__ DP, const float2* __restrict__ OP,
    const float* __restrict__ dscale,
    const float* __restrict__ offv_t, const double* __restrict__ gvec, double* __restrict__ xout,
    float* __restrict__ R, float* __restrict__ PA, float* __restrict__ PB,
    float* __restrict__ Dv, float* __restrict__ XH, float* __restrict__ XL,
    float* __restrict__ GH, float* __restrict__ GL, double rtol, int32_t max_iter,
    int32_t* __restrict__ iters, PcgStatus* __restrict__ status, int g32,
    double* __restrict__ gnout) {
  __shared__ BatchShared sh;
  const int32_t nv = g.nv;
  const int64_t ne2 = 2 * (int64_t)g.ne;
  const int64_t nsg = (S + kSG - 1) / kSG;
  const int64_t n_items = (int64_t)L * nsg;
  const int hh = threadIdx.x & 1;            // half row: samples 4 hh .. 4 hh + 3
  const int32_t vs = threadIdx.x >> 1;       // vertex lane
  const int32_t* __restrict__ nbr = g.adj_nbr;
  const double rtol2 = rtol * rtol;
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int64_t l = L - 1 - item / nsg;  // largest shifts first (longest solves)
    const int64_t s0 = (item % nsg) * kSG;
    const float2* __restrict__ Dp = DP + l * nv;
    const float2* __restrict__ Op = OP + l * ne2;
    const float* __restrict__ Ds = dscale + l * nv;
    const float* __restrict__ Ot = offv_t + l * ne2;
    const int64_t base = (l * nsg + (item % nsg)) * (int64_t)nv * kSG + 4 * hh;
    float* __restrict__ r = R + base;
    float* __restrict__ pa = PA + base;
    float* __restrict__ pb = PB + base;
    float* __restrict__ dv = Dv + base;
    float* __restrict__ xh = XH + base;
    float* __restrict__ xl = XL + base;
    float* __restrict__ gh = GH + base;
    float* __restrict__ gl = GL + base;
    // this thread's 4 samples: FP64 rows of g and x (row i at + i nv; only
    // the first nlive exist)
    const int64_t sfirst = s0 + 4 * hh;
    const int nlive = (int)(S - sfirst < 0 ? 0 : (S - sfirst > 4 ? 4 : S - sfirst));
    const double* __restrict__ g0 = g32 ? nullptr : gvec + (l * S + (nlive > 0 ? sfirst : 0)) * nv;
    double* __restrict__ x0 = xout + (l * S + (nlive > 0 ? sfirst : 0)) * nv;
#define GS(i) (g0 + (int64_t)(i) * nv)
#define XS(i) (x0 + (int64_t)(i) * nv)
#define LIVE(i) ((i) < nlive)

    // ---- ||g||^2, ||D^-1/2 g||^2 (FP64; from the FP32 g in gh: FP32 pair sums)
    {
      double out[2] = {0.0, 0.0};
      if (g32) {
        Acc4<2> a2;
        a2.init();
        for (int32_t v = vs; v < nv; v += kVP) {
          const float dsv = Ds[v];
          const float4 g4 = ld4(gh + (int64_t)v * kSG);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float gv = LIVE(i) ? get(g4, i) : 0.f, sv = gv * dsv;
            a2.f[i][0] = fmaf(gv, gv, a2.f[i][0]);
            a2.f[i][1] = fmaf(sv, sv, a2.f[i][1]);
          }
          a2.tick();
        }
        group_sum<2>(a2, sh, out);
      } else {
      double a[4][2] = {};
      for (int32_t v = vs; v < nv; v += kVP) {
        const double dsv = (double)Ds[v];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const double gv = LIVE(i) ? GS(i)[v] : 0.0;
          const double sv = gv * dsv;
          a[i][0] = fma(gv, gv, a[i][0]);
          a[i][1] = fma(sv, sv, a[i][1]);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int o = 2; o < 32; o <<= 1) a[i][k] += __shfl_xor_sync(kFull, a[i][k], o);
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      if (lane < 2) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k = 0; k < 2; ++k) sh.red[warp][4 * lane + i][k] = a[i][k];
      }
      __syncthreads();
      if (threadIdx.x < kSG) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int w = 0; w < kWarps; ++w) out[k] += sh.red[w][threadIdx.x][k];
      }
      }
      if (threadIdx.x < kSG) {
        SampleState& q = sh.st[threadIdx.x];
        const bool lv = s0 + threadIdx.x < S;
        q.bad = lv && (!isfinite(out[0]) || !isfinite(out[1]));
        q.done = !lv || q.bad || !(out[0] > 0.0) || !(out[1] > 0.0);
        q.gn = q.done ? 0.0 : sqrt(out[0]);
        q.inv_g = q.done ? 0.0 : 1.0 / q.gn;
        if (g32 && !q.done) {
          // g~ = g fl32(1 / ||g||) exactly as a pair; ||g|| the exact inverse
          // of that factor, so that x = ||g|| x~ solves S x = g
          const float ivf = (float)q.inv_g;
          if (!(ivf >= 1.17549435e-38f) || !isfinite(ivf)) {
            q.bad = q.done = 1;
          } else {
            q.inv_g = (double)ivf;
            q.gn = 1.0 / (double)ivf;
          }
        }
        // the inner FP32 solve runs on r = D^-1/2 r~ ||g|| / rho, O(1) whatever
        // the node's scale: rho = ||D^-1/2 g|| first, then the estimate of the
        // refinement residual's norm from the previous inner solve
        q.rho = q.done ? 1.0 : sqrt(out[1]);
        q.rz0 = q.done ? 0.0 : out[1] / (q.rho * q.rho);
        q.scl = q.done ? 0.f : (float)(q.gn / q.rho);
        q.inner_e = kInnerRtol;
        q.it = 0;
        q.cg = 0;
      }
      __syncthreads();
      // ---- g~ = g / ||g|| as FP32 pairs, x~ = 0, r = D^-1/2 g~ ||g|| / rho
      bool dn[4];
      double ivg[4];
      float sc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const SampleState& q = sh.st[4 * hh + i];
        dn[i] = q.done;
        ivg[i] = q.inv_g;
        sc[i] = q.scl;
      }
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int32_t v = vs; v < nv; v += kVP) {
        const float dsv = Ds[v];
        float hv[4], lv[4], rv[4];
        const int64_t iv = (int64_t)v * kSG;
        if (g32) {
          const float4 g4 = ld4(gh + iv);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float gv = dn[i] ? 0.f : get(g4, i), ivf = (float)ivg[i];
            hv[i] = gv * ivf;
            lv[i] = fmaf(gv, ivf, -hv[i]);  // g ivf = hv + lv exactly
            rv[i] = (hv[i] * sc[i]) * dsv;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const double gt = dn[i] ? 0.0 : GS(i)[v] * ivg[i];
            hv[i] = __double2float_rn(gt);
            lv[i] = __double2float_rn(gt - (double)hv[i]);
            rv[i] = (hv[i] * sc[i]) * dsv;
          }
        }
        st4(gh + iv, make_float4(hv[0], hv[1], hv[2], hv[3]));
        st4(gl + iv, make_float4(lv[0], lv[1], lv[2], lv[3]));
        st4(xh + iv, z4);
        st4(xl + iv, z4);
        st4(r + iv, make_float4(rv[0], rv[1], rv[2], rv[3]));
      }
      __syncthreads();
    }

    for (int32_t round = 0; round <= max_iter; ++round) {
      if (round > 0) {
        // ---- refinement residual r~ = g~ - S x~ in FP32-pair arithmetic;
        // stored r = D^-1/2 r~ ||g|| / rho
        bool dn[4];
        float sc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const SampleState& q = sh.st[4 * hh + i];
          dn[i] = q.done;
          sc[i] = q.scl;
        }
        Acc4<2> a;
        a.init();
        int4 ea_n[kU];
        int2 eb_n[kU];
        load_ell(ell, vs, nv, ea_n, eb_n);
        for (int32_t v = vs; v < nv; v += kVP) {
          if (threadIdx.x == 0) {  // rows of x~ and g~ kPF steps ahead
            prefetch_rows(xh, v, nv);
            prefetch_rows(xl, v, nv);
            prefetch_rows(gh, v, nv);
            prefetch_rows(gl, v, nv);
          }
          int4 ea[kU];
          int2 eb[kU];
          ea[0] = ea_n[0];
          eb[0] = eb_n[0];
          load_ell(ell, v + kVP, nv, ea_n, eb_n);  // the next step's records
          const int32_t k0 = eb[0].x, deg = eb[0].y;
          const int32_t wl[4] = {ea[0].x, ea[0].y, ea[0].z, ea[0].w};
          const int64_t iv = (int64_t)v * kSG;
          const float2 dp = Dp[v];
          const float dsv = Ds[v];
          const float4 xh0 = ld4(xh + iv), xl0 = ld4(xl + iv);
          const float4 g0h = ld4(gh + iv), g0l = ld4(gl + iv);
          float s4[4], c4[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            s4[i] = get(g0h, i);
            c4[i] = get(g0l, i);
            ff_sub_prod(s4[i], c4[i], dp.x, dp.y, get(xh0, i), get(xl0, i));
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (j < deg) {
              const float2 op = Op[k0 + j];
              const int64_t w = (int64_t)wl[j] * kSG;
              const float4 wh = ld4(xh + w), wlo = ld4(xl + w);
#pragma unroll
              for (int i = 0; i < 4; ++i)
                ff_sub_prod(s4[i], c4[i], op.x, op.y, get(wh, i), get(wlo, i));
            }
          }
          for (int32_t k = k0 + 4; k < k0 + deg; ++k) {
            const float2 op = Op[k];
            const int64_t w = (int64_t)nbr[k] * kSG;
            const float4 wh = ld4(xh + w), wlo = ld4(xl + w);
#pragma unroll
            for (int i = 0; i < 4; ++i)
              ff_sub_prod(s4[i], c4[i], op.x, op.y, get(wh, i), get(wlo, i));
          }
          float sv4[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float rel = dn[i] ? 0.f : s4[i] + c4[i];
            sv4[i] = (rel * sc[i]) * dsv;
            a.f[i][0] = fmaf(rel, rel, a.f[i][0]);
            a.f[i][1] = fmaf(sv4[i], sv4[i], a.f[i][1]);
          }
          a.tick();
          st4(r + iv, make_float4(sv4[0], sv4[1], sv4[2], sv4[3]));
        }
        double out[2] = {0.0, 0.0};
        group_sum<2>(a, sh, out);
        if (threadIdx.x < kSG) {
          SampleState& q = sh.st[threadIdx.x];
          if (!q.done) {
            if (!isfinite(out[0]) || !isfinite(out[1])) {
              q.bad = q.done = 1;
            } else if (out[0] <= rtol2) {
              q.done = 1;
            } else {
              q.rz0 = out[1];
              q.inner_e = fmax(kInnerRtol, 0.1 * sqrt(rtol2 / out[0]));
            }
          }
        }
      }
      // start an inner CG on the scaled system from d = 0, p = r
      int cgj = 0;
      if (threadIdx.x < kSG) {
        SampleState& q = sh.st[threadIdx.x];
        q.cg = !q.done && q.it < max_iter && q.rz0 > 0.0;
        q.rz = q.rz0;
        q.best = q.rz0;
        q.stop2 = q.inner_e * q.inner_e * q.rz0;
        q.since = 0;
        q.has_d = 0;
        q.first = 1;
        q.bf = 0.f;
        cgj = q.cg;
      }
      if (!__syncthreads_or(cgj)) break;
      for (int32_t inner = 0; inner < max_iter; ++inner) {
        bool cg[4], fs[4], any = false;
        float bf[4];
        const bool fst = sh.st[4 * hh].first;  // the group's samples start together
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const SampleState& q = sh.st[4 * hh + i];
          cg[i] = q.cg;
          fs[i] = q.first || !q.cg;
          bf[i] = q.bf;
          any |= cg[i];
        }
        const float* pold = (inner & 1) ? pb : pa;
        float* pnew = (inner & 1) ? pa : pb;
        // ---- pass A: p' = r + beta p (p' = r at the start), q = S p', p'.q
        {
          Acc4<1> a;
          a.init();
          if (any) {
            const float4 bf4 = make_float4(bf[0], bf[1], bf[2], bf[3]);
            // p' of vertex w from its r and old p
            auto pnext = [&](int64_t w, float4 rw) -> float4 {
              return fst ? rw : sel4(fs, rw, fma4(bf4, ld4(pold + w), rw));
            };
            int4 ea_n[kU];
            int2 eb_n[kU];
            load_ell(ell, vs, nv, ea_n, eb_n);
            for (int32_t v0 = vs; v0 < nv; v0 += kU * kVP) {
              if (threadIdx.x == 0) {  // rows of r and p kPF steps ahead (hh = 0 here)
                prefetch_rows(r, v0, nv);
                if (!fst) prefetch_rows(pold, v0, nv);
              }
              // this step's neighbour records, loaded one step earlier; the
              // next step's requested now
              int4 ea[kU];
              int2 eb[kU];
#pragma unroll
              for (int u = 0; u < kU; ++u) ea[u] = ea_n[u], eb[u] = eb_n[u];
              load_ell(ell, v0 + kU * kVP, nv, ea_n, eb_n);
#pragma unroll
              for (int u = 0; u < kU; ++u) {
                const int32_t v = v0 + u * kVP;
                if (v >= nv) break;
                const int32_t k0 = eb[u].x, deg = eb[u].y;
                const int32_t wl[4] = {ea[u].x, ea[u].y, ea[u].z, ea[u].w};
                const float4 pv = pnext((int64_t)v * kSG, ld4(r + (int64_t)v * kSG));
                float4 q = pv;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  if (i < deg) {
                    const int64_t w = (int64_t)wl[i] * kSG;
                    q = fma1(Ot[k0 + i], pnext(w, ld4(r + w)), q);
                  }
                }
                for (int32_t k = k0 + 4; k < k0 + deg; ++k) {
                  const int64_t w = (int64_t)nbr[k] * kSG;
                  q = fma1(Ot[k], pnext(w, ld4(r + w)), q);
                }
                st4(pnew + (int64_t)v * kSG, pv);
#pragma unroll
                for (int i = 0; i < 4; ++i) a.f[i][0] = fmaf(get(pv, i), get(q, i), a.f[i][0]);
              }
              a.tick();
            }
          }
          double out[1] = {0.0};
          group_sum<1>(a, sh, out);
          if (threadIdx.x < kSG) {
            SampleState& q = sh.st[threadIdx.x];
            q.af = 0.f;
            if (q.cg) {
              const double pq = out[0];
              if (!isfinite(pq)) {
                q.bad = q.done = 1;
                q.cg = 0;
              } else if (!(pq > 0.0)) {
                q.cg = 0;  // p vanished: the FP32 recurrence is at its floor
              } else {
                q.af = (float)(q.rz / pq);
              }
            }
          }
          __syncthreads();
        }
        // ---- pass B: q = S p' again, d += alpha p', r -= alpha q, r.r
        {
          bool hd[4];
          float af[4];
          any = false;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const SampleState& q = sh.st[4 * hh + i];
            cg[i] = q.cg;
            hd[i] = q.has_d;
            af[i] = cg[i] ? q.af : 0.f;
            any |= cg[i];
          }
          const float4 af4 = make_float4(af[0], af[1], af[2], af[3]);
          const float4 naf4 = make_float4(-af[0], -af[1], -af[2], -af[3]);
          Acc4<1> a;
          a.init();
          if (any) {
            int4 ea_n[kU];
            int2 eb_n[kU];
            load_ell(ell, vs, nv, ea_n, eb_n);
            for (int32_t v0 = vs; v0 < nv; v0 += kU * kVP) {
              if (threadIdx.x == 0) {  // rows of p', d and r kPF steps ahead
                prefetch_rows(pnew, v0, nv);
                prefetch_rows(dv, v0, nv);
                prefetch_rows(r, v0, nv);
              }
              int4 ea[kU];
              int2 eb[kU];
#pragma unroll
              for (int u = 0; u < kU; ++u) ea[u] = ea_n[u], eb[u] = eb_n[u];
              load_ell(ell, v0 + kU * kVP, nv, ea_n, eb_n);
#pragma unroll
              for (int u = 0; u < kU; ++u) {
                const int32_t v = v0 + u * kVP;
                if (v >= nv) break;
                const int32_t k0 = eb[u].x, deg = eb[u].y;
                const int32_t wl[4] = {ea[u].x, ea[u].y, ea[u].z, ea[u].w};
                const int64_t iv = (int64_t)v * kSG;
                const float4 pv = ld4(pnew + iv);
                float4 q = pv;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                  if (i < deg) q = fma1(Ot[k0 + i], ld4(pnew + (int64_t)wl[i] * kSG), q);
                for (int32_t k = k0 + 4; k < k0 + deg; ++k)
                  q = fma1(Ot[k], ld4(pnew + (int64_t)nbr[k] * kSG), q);
                const float4 d0 = ld4(dv + iv);
                const float4 r0 = ld4(r + iv);
                const float4 dn = fma4(af4, pv, make_float4(hd[0] ? d0.x : 0.f, hd[1] ? d0.y : 0.f,
                                                            hd[2] ? d0.z : 0.f, hd[3] ? d0.w : 0.f));
                const float4 rn = fma4(naf4, q, r0);
                st4(dv + iv, sel4(cg, dn, d0));
                st4(r + iv, rn);
#pragma unroll
                for (int i = 0; i < 4; ++i) a.f[i][0] = fmaf(get(rn, i), get(rn, i), a.f[i][0]);
              }
              a.tick();
            }
          }
          double out[1] = {0.0};
          group_sum<1>(a, sh, out);
          int cgj2 = 0;
          if (threadIdx.x < kSG) {
            SampleState& q = sh.st[threadIdx.x];
            q.first = 0;
            if (q.cg) {
              q.has_d = 1;
              ++q.it;
              const double rr = out[0];
              if (!isfinite(rr)) {
                q.bad = q.done = 1;
                q.cg = 0;
              } else {
                const double rz_prev = q.rz;
                q.rz = rr;
                if (rr <= q.stop2) {
                  q.cg = 0;
                } else {
                  if (rr < 0.98 * q.best) {
                    q.best = rr;
                    q.since = 0;
                  } else if (++q.since >= 32) {
                    q.cg = 0;  // the FP32 recurrence has reached its rounding floor
                  }
                  q.bf = (float)(rr / rz_prev);
                  if (q.it >= max_iter) q.cg = 0;
                }
              }
            }
            cgj2 = q.cg;
          }
          if (!__syncthreads_or(cgj2)) break;
        }
      }
      // ---- x~ += (rho / ||g||) D^-1/2 d for the samples that ran a correction
      // this round (FP32-pair update)
      {
        bool up[4], any = false;
        float xs[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const SampleState& q = sh.st[4 * hh + i];
          up[i] = q.has_d && !q.bad;
          xs[i] = up[i] ? (float)(q.rho * q.inv_g) : 0.f;
          any |= up[i];
        }
        if (any) {
          for (int32_t v = vs; v < nv; v += kVP) {
            const int64_t iv = (int64_t)v * kSG;
            const float4 d4 = ld4(dv + iv);
            float4 h4 = ld4(xh + iv), l4 = ld4(xl + iv);
            const float dsv = Ds[v];
            float hv[4] = {h4.x, h4.y, h4.z, h4.w}, lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (up[i]) ff_add(hv[i], lv[i], (xs[i] * dsv) * get(d4, i));
            st4(xh + iv, make_float4(hv[0], hv[1], hv[2], hv[3]));
            st4(xl + iv, make_float4(lv[0], lv[1], lv[2], lv[3]));
          }
        }
      }
      __syncthreads();  // x~ complete, every thread done with the state
      if (threadIdx.x < kSG) {
        SampleState& q = sh.st[threadIdx.x];
        if (q.has_d && !q.bad) {
          q.rho *= sqrt(fmax(q.rz, 1e-24 * q.rz0));
          q.scl = (float)(q.gn / q.rho);
        }
      }
      __syncthreads();
    }
    // ---- x = ||g|| (x~hi + x~lo) in FP64; or only ||g|| per system, from
    // which pcg_batch_out_kernel forms the recovery's weighted values
    if (gnout) {
      if (threadIdx.x < kSG && s0 + threadIdx.x < S)
        gnout[l * S + s0 + threadIdx.x] = sh.st[threadIdx.x].gn;
    } else {
      double gn[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) gn[i] = sh.st[4 * hh + i].gn;
      for (int32_t v = vs; v < nv; v += kVP) {
        const int64_t iv = (int64_t)v * kSG;
        const float4 h4 = ld4(xh + iv), l4 = ld4(xl + iv);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (LIVE(i)) XS(i)[v] = gn[i] * ((double)get(h4, i) + (double)get(l4, i));
      }
    }
    if (threadIdx.x < kSG && s0 + threadIdx.x < S) {
      const SampleState& q = sh.st[threadIdx.x];
      const int64_t sys = l * S + s0 + threadIdx.x;
      iters[sys] = q.it;
      atomicAdd(&status->iters_total, (unsigned long long)q.it);
      atomicMax(&status->iters_max, q.it);
      if (q.bad) atomicAdd(&status->numeric_flag, 1);
      else if (!q.done) atomicAdd(&status->n_unconverged, 1);
    }
    __syncthreads();
  }
}

#undef GS
#undef XS
#undef LIVE

// xw[l][v][s] = w_l ||g||_ls (x~hi + x~lo)[l][s / 8][v][s % 8] in FP32: thread
// per (l, v, four samples), consecutive threads on consecutive samples, so the
// writes are coalesced and the reads whole 16-byte pieces of the sample rows.
__global__ void __launch_bounds__(256)
    pcg_batch_out_kernel(int32_t nv, int32_t L, int64_t S, const float* __restrict__ XH,
                         const float* __restrict__ XL, const double* __restrict__ gn,
                         const double* __restrict__ weight, float* __restrict__ xw) {
  const int64_t nq = (S + 3) / 4, nsg = (S + kSG - 1) / kSG;
  const int64_t n = (int64_t)L * nv * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t % nq, lv = t / nq;
    const int64_t v = lv % nv, l = lv / nv;
    const int64_t s = 4 * q;
    const int64_t src = ((l * nsg + s / kSG) * nv + v) * kSG + (s % kSG);
    const float4 h = ld4(XH + src), lo = ld4(XL + src);
    const double w = weight[l];
    const float y[4] = {h.x + lo.x, h.y + lo.y, h.z + lo.z, h.w + lo.w};
    float* o = xw + lv * S + s;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (s + i < S) o[i] = (float)(w * gn[l * S + s + i]) * y[i];
  }
}

// Vectors of the batched layout need [L][ceil(S / 8) * 8][nv] floats each.
int64_t pcg_batch_padded_samples(int64_t S) { return (S + kSG - 1) / kSG * kSG; }

// diag and offv (FP64) are read through their FP32-pair copies pp.dp, pp.op.
void launch_pcg_batch(const DevGraph& g, const int4* ell, int32_t L, int64_t S, const double* diag,
                      const double* offv, const float* dscale, const float* offv_t,
                      const double* gvec, double* x, float* R, float* PA, float* PB, float* Dv,
                      const PcgPairs& pp, double rtol, int32_t max_iter, int32_t* iters,
                      PcgStatus* status, cudaStream_t st) {
  (void)diag;
  (void)offv;
  const int64_t items = (int64_t)L * ((S + kSG - 1) / kSG);
  if (items <= 0) return;
  const int blocks = (int)(items < (int64_t)1 << 30 ? items : (int64_t)1 << 30);
  pcg_batch_kernel<<<blocks, kBT, 0, st>>>(g, ell, L, S, pp.dp, pp.op, dscale, offv_t, gvec, x, R,
                                           PA, PB, Dv, pp.xh, pp.xl, pp.gh, pp.gl, rtol, max_iter,
                                           iters, status, pp.g32 ? 1 : 0,
                                           pp.xw ? pp.gn : nullptr);
  if (pp.xw) {
    const int64_t n = (int64_t)L * g.nv * ((S + 3) / 4);
    const int64_t blocks = (n + 255) / 256 < (int64_t)sm_count() * 32 ? (n + 255) / 256
                                                                        : (int64_t)sm_count() * 32;
    pcg_batch_out_kernel<<<(int)blocks, 256, 0, st>>>(g.nv, L, S, pp.xh, pp.xl, pp.gn, pp.weight,
                                                      pp.xw);
  }
}

}  // namespace grf
