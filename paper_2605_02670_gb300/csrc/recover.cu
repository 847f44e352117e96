// Fused interior recovery + quadrature sum (Eq. internal_recovery, Sec. 3
// Phase 5) with the edge interior held in registers.
//
// For every node l the interior values of edge e solve
//   T_l x = (w_l / c_l) b_I + w_l u_a e_1 + w_l u_b e_m,
//   T_l = tridiag(-1, 2 + delta_l, -1),  c_l = gamma_l / h_e,
// and U_I = sum_l x^(l). A unit of work is (edge, group of SG samples). The
// unit's m interior nodes are split into contiguous segments of B nodes, one
// per lane of NW warps, and stay in registers for all L nodes: the noise is
// read once and the field written once.
//
// Thomas forward elimination y_K = r_K + y_{K-1} / p_{K-1} and back
// substitution x_K = (y_K + x_{K+1}) / p_K are first-order affine recurrences;
// each lane runs them on its segment from a zero carry, the carries are found
// by a scan of the composed affine maps across lanes (warp shuffles, shared
// memory across warps), and each lane then adds carry x (product of 1/p) to its
// values.
//
// Pivots p_K = 1 + q_K: with 2 + delta = 2 cosh(theta) the elimination pivots
// of T are p_K = sinh((K+1) theta) / sinh(K theta), so
//   q_K = delta / 2 + sinh(theta) coth(K theta)
// with no subtraction. A lane evaluates this once at the start of its segment
// and continues with q_{K+1} = delta + q_K / (1 + q_K) (the same excess
// recurrence the sequential sweep uses), which is contracting, so the start
// error does not grow.
//
// The sum over nodes: partial sums in the sweep precision over `group`
// consecutive nodes, added into an FP64 accumulator held in shared memory.
//
// SG trades registers for shared work: pivots and the scans' multipliers are
// computed once per lane for SG samples, while fewer samples per lane leave
// room for more resident warps. It is a launch parameter picked by measurement.
#include <type_traits>

#include "grf_internal.h"

namespace grf {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// FP32 pivots use the SFU reciprocal (relative error a few 1e-8): the sweeps
// contract, so pivot errors of that size stay at that size.
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float quot(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double quot(double a, double b) { return a / b; }
// K theta from which coth(K theta) = 1 in the working precision (2 exp(-2 K
// theta) below half an ulp): the pivots of such nodes are the fixed point.
// SG consecutive values of a shared-memory row (aligned to SG * sizeof(T)).
template <typename T, int SG>
__device__ __forceinline__ void load_vec(const T* p, T (&v)[SG]) {
  if constexpr (std::is_same<T, float>::value && SG == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (std::is_same<T, float>::value && SG == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  } else if constexpr (std::is_same<T, double>::value && SG == 2) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x; v[1] = t.y;
  } else {
#pragma unroll
    for (int s = 0; s < SG; ++s) v[s] = p[s];
  }
}

template <typename T>
constexpr T kConvTheta = sizeof(T) == 4 ? (T)9 : (T)19;
__device__ __forceinline__ float tanh_t(float x) { return tanhf(x); }
__device__ __forceinline__ double tanh_t(double x) { return tanh(x); }

// Inclusive composition of affine maps y -> R + A y across the lanes of a warp.
// forward: lane i ends with f_i o f_{i-1} o ... o f_0;
// backward: lane i ends with f_i o f_{i+1} o ... o f_31.
// Only the first SPAN lanes need the result (lanes from SPAN on hold the
// identity when SPAN < 32).
template <typename T, int SG, bool kForward, int SPAN = 32>
__device__ __forceinline__ void warp_scan(T& a, T (&r)[SG], int lane) {
#pragma unroll
  for (int d = 1; d < SPAN; d <<= 1) {
    T ap, rp[SG];
    if (kForward) {
      ap = __shfl_up_sync(kFull, a, d);
#pragma unroll
      for (int s = 0; s < SG; ++s) rp[s] = __shfl_up_sync(kFull, r[s], d);
    } else {
      ap = __shfl_down_sync(kFull, a, d);
#pragma unroll
      for (int s = 0; s < SG; ++s) rp[s] = __shfl_down_sync(kFull, r[s], d);
    }
    const bool take = kForward ? (lane >= d) : (lane + d < 32);
    if (take) {
#pragma unroll
      for (int s = 0; s < SG; ++s) r[s] = fma(a, rp[s], r[s]);
      a = a * ap;
    }
  }
}

// Carry into this lane: the value at the end of the previous lane (forward) or
// at the start of the next lane (backward), given the lane's own map (a, r).
// NW > 1 combines warp totals through shared memory.
template <typename T, int SG, bool kForward, int NW>
__device__ __forceinline__ void lane_carry(T a, const T (&r)[SG], int lane, int wi,
                                           T (*sh_a)[NW], T (*sh_r)[NW][SG], T (&carry)[SG]) {
  T ia = a, ir[SG];
#pragma unroll
  for (int s = 0; s < SG; ++s) ir[s] = r[s];
  warp_scan<T, SG, kForward>(ia, ir, lane);
  // exclusive: the neighbour's inclusive result
  const bool edge_lane = kForward ? (lane == 0) : (lane == 31);
  T ea = kForward ? __shfl_up_sync(kFull, ia, 1) : __shfl_down_sync(kFull, ia, 1);
  T er[SG];
#pragma unroll
  for (int s = 0; s < SG; ++s)
    er[s] = kForward ? __shfl_up_sync(kFull, ir[s], 1) : __shfl_down_sync(kFull, ir[s], 1);
  if (edge_lane) {
    ea = (T)1;
#pragma unroll
    for (int s = 0; s < SG; ++s) er[s] = (T)0;
  }
  T win[SG];
#pragma unroll
  for (int s = 0; s < SG; ++s) win[s] = (T)0;
  if constexpr (NW > 1) {
    // One barrier per direction and node: the forward and backward totals
    // live in separate rows, and a row is rewritten only after the other
    // direction's barrier, which every warp passes after its last read.
    const int tot_lane = kForward ? 31 : 0;
    const int dir = kForward ? 0 : 1;
    if (lane == tot_lane) {
      sh_a[dir][wi] = ia;
#pragma unroll
      for (int s = 0; s < SG; ++s) sh_r[dir][wi][s] = ir[s];
    }
    __syncthreads();
    // lane j < NW takes warp j's total, the other lanes the identity; one scan
    // over them gives every warp the composition of the warps before (after) it
    T ta = (T)1, tr[SG];
#pragma unroll
    for (int s = 0; s < SG; ++s) tr[s] = (T)0;
    if (lane < NW) {
      ta = sh_a[dir][lane];
#pragma unroll
      for (int s = 0; s < SG; ++s) tr[s] = sh_r[dir][lane][s];
    }
    warp_scan<T, SG, kForward, NW>(ta, tr, lane);
    const int src = kForward ? wi - 1 : wi + 1;
    const bool none = kForward ? wi == 0 : wi == NW - 1;
#pragma unroll
    for (int s = 0; s < SG; ++s) {
      const T t = __shfl_sync(kFull, tr[s], src & 31);
      win[s] = none ? (T)0 : t;
    }
  }
#pragma unroll
  for (int s = 0; s < SG; ++s) carry[s] = fma(ea, win[s], er[s]);
}

// Dynamic shared memory per CTA: the FP64 node sums [warp][B*SG][32], and for
// kRbSmem the unit's noise [warp][B][32][SG].
template <typename T, int B, int NW, int UPC, bool kRbSmem, int SG>
constexpr size_t seg_smem_bytes() {
  return (size_t)UPC * NW * B * SG * 32 * (sizeof(double) + (kRbSmem ? sizeof(T) : 0));
}

template <typename T, int B, int NW, int UPC, bool kRbSmem, int SG>
__global__ void __launch_bounds__(32 * NW * UPC)
    recover_seg_kernel(DevGraph g, int32_t L, int64_t S, const int32_t* __restrict__ edges,
                       int32_t n_edges, const T* __restrict__ b,
                       const SweepParams<T>* __restrict__ prm, const T* __restrict__ xw,
                       void* __restrict__ out, int out_f64, int group) {
  __shared__ T sh_a[2][NW];
  __shared__ T sh_r[2][NW][SG];
  extern __shared__ __align__(16) unsigned char dyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ul = warp / NW, wi = warp % NW;
  double(*acc)[32] = reinterpret_cast<double(*)[32]>(dyn) + (size_t)warp * B * SG;
  T* rbs = reinterpret_cast<T*>(dyn + (size_t)UPC * NW * B * SG * 32 * sizeof(double)) +
           (size_t)warp * B * 32 * SG;
  const int64_t nsg = (S + SG - 1) / SG;
  const int64_t n_units = (int64_t)n_edges * nsg;
  // all warps of a CTA take the same number of trips (NW > 1 uses __syncthreads)
  const int64_t trips = (n_units + (int64_t)gridDim.x * UPC - 1) / ((int64_t)gridDim.x * UPC);
  for (int64_t trip = 0; trip < trips; ++trip) {
    const int64_t unit = (trip * gridDim.x + blockIdx.x) * UPC + ul;
    const bool live = unit < n_units;
    const int32_t e = live ? edges[unit / nsg] : 0;
    const int64_t s0 = live ? (unit % nsg) * SG : 0;
    const int32_t m = live ? g.nel[e] - 1 : 0;
    const int64_t off = live ? g.ioff[e] : 0;
    const int32_t va = live ? g.eu[e] : 0, vb = live ? g.ev[e] : 0;
    const int K0 = (wi * 32 + lane) * B + 1;  // 1-based first node of this lane
    T rb[kRbSmem ? 1 : B][SG];
#pragma unroll
    for (int k = 0; k < B; ++k) {
#pragma unroll
      for (int s = 0; s < SG; ++s) {
        const bool ok = (K0 + k <= m) && (s0 + s < S);
        const T v = ok ? b[(g.nv + off + K0 + k - 1) * S + s0 + s] : (T)0;
        if (kRbSmem)
          rbs[(k * 32 + lane) * SG + s] = v;
        else
          rb[kRbSmem ? 0 : k][s] = v;
        acc[k * SG + s][lane] = 0.0;
      }
    }
    T accf[B][SG];
#pragma unroll
    for (int k = 0; k < B; ++k)
#pragma unroll
      for (int s = 0; s < SG; ++s) accf[k][s] = (T)0;

    // the boundary values enter only the lanes holding node 1 (x_a) and node m (x_b)
    const bool has1 = live && K0 == 1;
    const bool hasm = live && K0 <= m && m < K0 + B;
    const int km = m - K0;  // slot of node m in this lane when hasm
    const SweepParams<T>* pe = prm + e;
    const T* xap = xw + (int64_t)va * S + s0;
    const T* xbp = xw + (int64_t)vb * S + s0;
    const int64_t xstep = (int64_t)g.nv * S;
    for (int32_t l = 0; l < L; ++l, pe += g.ne, xap += xstep, xbp += xstep) {
      const SweepParams<T> pr = *pe;
      const T dl = pr.delta, sc = pr.sc, shv = pr.sh, th = pr.theta;
      // The sweeps run on the right-hand side divided by sc (b + (x_a / sc) e_1 +
      // (x_b / sc) e_m); the factor sc is applied once, when summing over nodes.
      T xa[SG], xb[SG];
      if (has1 || hasm) {
        const T isc = rcp(sc);
#pragma unroll
        for (int s = 0; s < SG; ++s) {
          const bool ok = s0 + s < S;
          xa[s] = (has1 && ok) ? xap[s] * isc : (T)0;
          xb[s] = (hasm && ok) ? xbp[s] * isc : (T)0;
        }
      } else {
#pragma unroll
        for (int s = 0; s < SG; ++s) xa[s] = xb[s] = (T)0;
      }
      // pivots of this lane's nodes (rp[k] = 1 / p_{K0+k}) and of the node before
      T rp_prev, rp[B];
      if (K0 >= 2 && (T)(K0 - 1) * th >= kConvTheta<T>) {
        // every node of the lane is at the fixed point p* = 1 + delta / 2 + sinh(theta)
        const T rps = rcp((T)1 + (T)0.5 * dl + shv);
        rp_prev = rps;
        if (hasm) {
#pragma unroll
          for (int k = 0; k < B; ++k) rp[k] = k <= km ? rps : (T)0;
        } else {
          const T r_ = K0 <= m ? rps : (T)0;
#pragma unroll
          for (int k = 0; k < B; ++k) rp[k] = r_;
        }
      } else {
        T q;
        if (K0 >= 2) {
          q = (T)0.5 * dl + quot(shv, tanh_t((T)(K0 - 1) * th));
          rp_prev = rcp((T)1 + q);
          q = dl + q * rp_prev;
        } else {
          rp_prev = (T)0;
          q = (T)1 + dl;
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const T r_ = rcp((T)1 + q);
          rp[k] = (K0 + k <= m) ? r_ : (T)0;
          q = dl + q * r_;
        }
      }
      if (K0 > m) rp_prev = (T)0;
      // forward elimination from a zero carry
      T y[B][SG];
#pragma unroll
      for (int k = 0; k < B; ++k) {
        T bv[SG];
        if (kRbSmem)
          load_vec<T, SG>(rbs + (k * 32 + lane) * SG, bv);
        else
#pragma unroll
          for (int s = 0; s < SG; ++s) bv[s] = rb[kRbSmem ? 0 : k][s];
#pragma unroll
        for (int s = 0; s < SG; ++s)
          y[k][s] = (k == 0) ? bv[s] + xa[s] : fma(rp[k - 1], y[k - 1][s], bv[s]);
      }
      T af = rp_prev;
#pragma unroll
      for (int k = 0; k < B - 1; ++k) af *= rp[k];
      T yin[SG];
      lane_carry<T, SG, true, NW>(af, y[B - 1], lane, wi, sh_a, sh_r, yin);
      {
        T c = rp_prev;
#pragma unroll
        for (int k = 0; k < B; ++k) {
          if (k > 0) c *= rp[k - 1];
#pragma unroll
          for (int s = 0; s < SG; ++s) y[k][s] = fma(c, yin[s], y[k][s]);
        }
      }
      // x_b enters at node m: y_m is used only by the back substitution there
      if (hasm) {
#pragma unroll
        for (int k = 0; k < B; ++k)
          if (k == km)
#pragma unroll
            for (int s = 0; s < SG; ++s) y[k][s] += xb[s];
      }
      // back substitution from a zero carry: x_K = (y_K + x_{K+1}) / p_K
#pragma unroll
      for (int k = B - 1; k >= 0; --k) {
#pragma unroll
        for (int s = 0; s < SG; ++s)
          y[k][s] = (k == B - 1) ? y[k][s] * rp[k] : (y[k][s] + y[k + 1][s]) * rp[k];
      }
      T ab = (T)1;
#pragma unroll
      for (int k = 0; k < B; ++k) ab *= rp[k];
      T xin[SG];
      lane_carry<T, SG, false, NW>(ab, y[0], lane, wi, sh_a, sh_r, xin);
      {
        T c = (T)1;
#pragma unroll
        for (int k = B - 1; k >= 0; --k) {
          c *= rp[k];
#pragma unroll
          for (int s = 0; s < SG; ++s) accf[k][s] = fma(sc, fma(c, xin[s], y[k][s]), accf[k][s]);
        }
      }
      if ((l + 1) % group == 0 || l + 1 == L) {
#pragma unroll
        for (int k = 0; k < B; ++k)
#pragma unroll
          for (int s = 0; s < SG; ++s) {
            acc[k * SG + s][lane] += (double)accf[k][s];
            accf[k][s] = (T)0;
          }
      }
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int K = K0 + k;
#pragma unroll
      for (int s = 0; s < SG; ++s) {
        if (live && K <= m && s0 + s < S) {
          const int64_t o = (s0 + s) * g.n + g.nv + off + K - 1;
          const double val = acc[k * SG + s][lane];
          if (out_f64)
            static_cast<double*>(out)[o] = val;
          else
            static_cast<float*>(out)[o] = (float)val;
        }
      }
    }
  }
}

int grid_for(int64_t units, int upc) {
  int64_t blocks = (units + upc - 1) / upc;
  if (blocks > sm_count() * 32) blocks = sm_count() * 32;
  return blocks < 1 ? 1 : (int)blocks;
}

template <typename T, int B, int NW, int SG>
void launch_bin(const DevGraph& g, int32_t L, int64_t S, const int32_t* edges, int32_t n,
                const T* b, const SweepParams<T>* prm, const T* xw, void* out, int out_f64,
                int group, cudaStream_t st) {
  if (n <= 0) return;
  constexpr int UPC = NW == 1 ? 4 : 1;
  constexpr bool kRbSmem = NW > 4;
  constexpr size_t smem = seg_smem_bytes<T, B, NW, UPC, kRbSmem, SG>();
  auto kern = recover_seg_kernel<T, B, NW, UPC, kRbSmem, SG>;
  // dynamic + static shared memory may pass the 48 KB default; the attribute is
  // per device, so it is set at every launch
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t units = (int64_t)n * ((S + SG - 1) / SG);
  kern<<<grid_for(units, UPC), 32 * NW * UPC, smem, st>>>(g, L, S, edges, n, b, prm, xw, out,
                                                        out_f64, group);
}

template <typename T, int SG>
int launch_all_bins(const DevGraph& g, int32_t L, int64_t S, const T* b,
                    const SweepParams<T>* prm, const T* xw, void* out, int out_f64,
                    const int32_t* bin_edges, const int32_t* bin_count, cudaStream_t st) {
  // partial sums over 32 consecutive nodes before each FP64 addition
  const int group = sizeof(T) == 4 ? 32 : (1 << 30);
  const int32_t* e = bin_edges;
  int n = 0;
#define GRF_BIN(i, B_, NW_)                                                                \
  launch_bin<T, B_, NW_, SG>(g, L, S, e, bin_count[i], b, prm, xw, out, out_f64, group, st); \
  n += bin_count[i] > 0;                                                                   \
  e += bin_count[i];
  if constexpr (sizeof(T) == 4) {
    GRF_BIN(0, 1, 1) GRF_BIN(1, 2, 1) GRF_BIN(2, 4, 1) GRF_BIN(3, 8, 1)
    GRF_BIN(4, 8, 2) GRF_BIN(5, 8, 4) GRF_BIN(6, 8, 8) GRF_BIN(7, 8, 16)
  } else {
    GRF_BIN(0, 1, 1) GRF_BIN(1, 2, 1) GRF_BIN(2, 4, 1) GRF_BIN(3, 4, 2)
    GRF_BIN(4, 4, 4) GRF_BIN(5, 4, 8) GRF_BIN(6, 4, 16)
  }
#undef GRF_BIN
  return n;
}

}  // namespace

// Bin table: bin i holds edges whose interior fits 32 * NW lanes x B nodes;
// longer edges go to the generic sequential kernel.
int recover_bins(bool fp64, int32_t* B_out, int32_t* NW_out) {
  static const int32_t bf[] = {1, 2, 4, 8, 8, 8, 8, 8};
  static const int32_t wf[] = {1, 1, 1, 1, 2, 4, 8, 16};
  static const int32_t bd[] = {1, 2, 4, 4, 4, 4, 4};
  static const int32_t wd[] = {1, 1, 1, 2, 4, 8, 16};
  const int n = fp64 ? 7 : 8;
  for (int i = 0; i < n; ++i) {
    B_out[i] = fp64 ? bd[i] : bf[i];
    NW_out[i] = fp64 ? wd[i] : wf[i];
  }
  return n;
}

template <typename T, typename OutT>
int launch_recover_bins(const DevGraph& g, int32_t L, int64_t S, const T* b,
                        const SweepParams<T>* prm, const T* xw, OutT* out,
                        const int32_t* bin_edges, const int32_t* bin_count, int sg,
                        cudaStream_t st) {
  const int f64 = sizeof(OutT) == 8;
  if constexpr (sizeof(T) == 4) {
    if (sg == 1)
      return launch_all_bins<T, 1>(g, L, S, b, prm, xw, out, f64, bin_edges, bin_count, st);
    if (sg == 2)
      return launch_all_bins<T, 2>(g, L, S, b, prm, xw, out, f64, bin_edges, bin_count, st);
    return launch_all_bins<T, 4>(g, L, S, b, prm, xw, out, f64, bin_edges, bin_count, st);
  } else {
    return launch_all_bins<T, 2>(g, L, S, b, prm, xw, out, f64, bin_edges, bin_count, st);
  }
}

#define GRF_INST(T, O)                                                                         \
  template int launch_recover_bins<T, O>(const DevGraph&, int32_t, int64_t, const T*,          \
                                         const SweepParams<T>*, const T*, O*, const int32_t*, \
                                         const int32_t*, int, cudaStream_t);
GRF_INST(float, float)
GRF_INST(float, double)
GRF_INST(double, double)
GRF_INST(double, float)
#undef GRF_INST

}  // namespace grf
