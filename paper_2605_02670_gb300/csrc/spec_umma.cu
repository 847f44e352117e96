// The two node contractions of the sine-basis edge-interior solves (Sec. 3,
// Phases 3 and 5 through the exact change of basis of the uniform lumped edge
// mesh) on the 5th-generation tensor cores.
//
// On edge e (m interior nodes, mesh width h) with the node constants
// delta_l = shift_l h^2, the mode shifts sig_j = 4 sin^2(pi (j+1) / (2 (m+1)))
// (j = 0 .. m-1) and eps_l = 1 (lumped mass) or 1 - delta_l / 6 (consistent
// mass), the interior eigenvalues of node l are (delta_l + sig_j eps_l) / eps_l.
// Both contractions are products with a matrix that is generated, not loaded:
//
//   end values (condensation), rows = nodes l, K = modes j:
//     O_l(s) = sum over even j of  A_lj phi_j bh_j(s),   E_l(s) = same over odd j,
//     A_lj = eps_l / (delta_l + sig_j eps_l);
//     g_a(l, s) += O + E,  g_b(l, s) += O - E   (the two end vertices of e);
//   coefficients (recovery), rows = modes j, K = nodes l:
//     C_j(s) = sum_l A'_jl eps_l X_l(s),   X = xa + xb (even j) or xa - xb (odd j),
//     A'_jl = 1 / (delta_l + sig_j eps_l),
//     D_j = sum_l sc_l A'_jl (FP32, by the thread that generates row j),
//     c_j(s) = D_j bh_j(s) + phi_j C_j(s), written over bh_j(s).
// Here phi_j = sqrt(2/(m+1)) sin(pi (j+1) / (m+1)), bh = Phi b_I the forward
// transform of the interior noise, xa_l / xb_l the weighted vertex values
// w_l u^(l) of the two end vertices and sc_l = w_l / c_l.
//
// Splitting the modes by parity makes each product a plain GEMM: the end-value
// K runs over the even modes into one accumulator and then over the odd modes
// into another; a coefficient unit takes 128 modes of one parity against that
// parity's right-hand side (xa + xb or xa - xb).
//
// Two CTAs of 256 threads per SM walk (edge, sample block, row block[, parity])
// units, so that one CTA's barriers and latencies overlap the other's work. A
// unit is a 128-row tile of A (UMMA M = 128) against a 64-wide K stage at a
// time, double-buffered: threads t and t + 128 generate the two halves of row
// t of A (32 reciprocals each, split into BF16 hi/lo, stored in the
// 128-byte-swizzled K-major layout) from per-unit tables laid out in K order,
// and the B tile of the next stage waits in registers while one thread issues
// the 12 MMAs of the current stage (4 K steps x 3 split products, FP32
// accumulators in tensor memory, N = the sample block of at most 32).
// Epilogues: the end values go to a per-edge buffer [e][end][s][l] (lanes on
// consecutive nodes, plain coalesced stores) and a gather over each vertex's
// incidences adds them into g, where FP64 atomics into the vertex-major g
// cost one scattered read-modify-write per value; the coefficients pass
// through a shared-memory tile so that the rows c_j are written with
// consecutive threads on consecutive samples, against bh rows fetched by
// cp.async when the unit starts.
// Every mbarrier wait is bounded: on a timeout the CTA raises the error flag,
// waits (bounded) for its MMAs, frees its tensor memory and stops.
#include "grf_internal.h"
#include "umma.cuh"

namespace grf {
namespace {

using namespace umma;

constexpr int kT = 256;                        // threads; t and t + 128 share row t of A
constexpr int kRows = 128;                     // A rows per unit (one UMMA tile)
constexpr int kK = 64;                         // K per stage
constexpr int kMaxSB = 32;                     // samples per unit (UMMA N)
constexpr uint32_t kATile = kRows * kK * 2;    // one BF16 plane of A: 16 KB
constexpr uint32_t kBPlane = kMaxSB * kK * 2;  // 4 KB
constexpr uint32_t kStage = 2 * kATile + 2 * kBPlane;  // A hi/lo, B hi/lo
constexpr uint32_t kBhTile = kRows * kMaxSB * 4;       // a coefficient unit's bh rows: 16 KB
constexpr int kMaxM = kSpecMaxM;               // modes of the sine-basis path
constexpr int kMaxKE = kMaxM + 2 * kK;         // K positions of the end values (both parities)
constexpr int kEndsRB = 2;                     // row blocks of 128 nodes per end-value unit
constexpr uint32_t kColsEnds = 2 * kEndsRB * 32;  // two accumulators of SB columns per block
constexpr int kMaxRB = (kMaxM / 2 + 127) / 128;  // row blocks of one parity's modes
constexpr uint32_t kColsCoef = kMaxRB * kMaxSB;   // one accumulator per row block
constexpr size_t kSmemLimit = 232448;          // 227 KB per CTA

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  const uint32_t a = smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

__device__ __forceinline__ float mode_shift(int32_t j, int32_t m) {
  const float sh = 2.f * sinpif((float)(j + 1) / (float)(2 * (m + 1)));
  return sh * sh;
}

// Shared bookkeeping of both kernels: two stage barriers, the tensor-memory
// slot, bounded waits and the teardown.
struct Pipe {
  uint64_t* mbar;
  uint32_t* tslot;
  uint32_t cols;
  uint32_t uses0, uses1;  // commits to each stage's barrier so far
  bool failed;

  __device__ uint32_t uses(int st) const { return st ? uses1 : uses0; }
  __device__ void bump(int st) {
    if (st)
      ++uses1;
    else
      ++uses0;
  }
  __device__ void init(unsigned char* at, uint32_t tmem_cols) {
    mbar = reinterpret_cast<uint64_t*>(at);
    tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    cols = tmem_cols;
    uses0 = uses1 = 0;
    failed = false;
    if (threadIdx.x == 0) {
      mbar_init(&mbar[0], 1);
      mbar_init(&mbar[1], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) tmem_alloc(tslot, cols);
    fence_before();
    __syncthreads();
    fence_after();
  }
  // before stage buffer st is written again: its previous MMAs are done
  __device__ bool acquire(int st) {
    const uint32_t n = uses(st);
    if (n > 0 && !mbar_wait(&mbar[st], (n - 1) & 1)) failed = true;
    failed = __syncthreads_or(failed);
    return !failed;
  }
  // after the last stage of a unit: every MMA of the unit is done
  __device__ bool drain(int last) {
    if (!mbar_wait(&mbar[last], (uses(last) - 1) & 1)) failed = true;
    failed = __syncthreads_or(failed);
    if (!failed) fence_after();
    return !failed;
  }
  __device__ void finish(PcgStatus* status) {
    if (failed) {
      if (threadIdx.x == 0) atomicAdd(&status->device_timeout, 1);
      if (uses0 > 0) mbar_wait(&mbar[0], (uses0 - 1) & 1);
      if (uses1 > 0) mbar_wait(&mbar[1], (uses1 - 1) & 1);
    }
    fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(*tslot, cols);
  }
};

// Chunk c (8 values) of row t of A in one stage: split and stored.
__device__ __forceinline__ void store_a_row(unsigned char* a_hi, unsigned char* a_lo, int t,
                                            int c, const float (&x)[8]) {
  uint4 hi, lo;
  split8(x, hi, lo);
  *reinterpret_cast<uint4*>(a_hi + swz(t, c)) = hi;
  *reinterpret_cast<uint4*>(a_lo + swz(t, c)) = lo;
}

__device__ __forceinline__ void store_b_row(unsigned char* b_hi, unsigned char* b_lo, int n,
                                            int c, const float (&x)[8]) {
  uint4 hi, lo;
  split8(x, hi, lo);
  *reinterpret_cast<uint4*>(b_hi + swz(n, c)) = hi;
  *reinterpret_cast<uint4*>(b_lo + swz(n, c)) = lo;
}

// The 12 MMAs of one stage into the accumulator at column col.
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint32_t col, unsigned char* a_hi,
                                            unsigned char* a_lo, unsigned char* b_hi,
                                            unsigned char* b_lo, uint32_t idesc, bool acc) {
  fence_after();
  mma_split_stage(tmem + col, sdesc(smem_u32(a_hi)), sdesc(smem_u32(a_lo)), sdesc(smem_u32(b_hi)),
                  sdesc(smem_u32(b_lo)), idesc, acc);
}

// ---------------------------------------------------------------- end values

template <bool kCons>
__global__ void __launch_bounds__(kT, 2)
    spec_ends_umma_kernel(DevGraph g, DevNodes nd, int64_t S, const int32_t* __restrict__ edges,
                          int32_t n_edges, const float* __restrict__ bhat,
                          double* __restrict__ gvec, float* __restrict__ ends, int32_t SB,
                          PcgStatus* __restrict__ status) {
  extern __shared__ unsigned char se_raw[];
  unsigned char* sm = align1024(se_raw);
  // two A buffers (hi and lo planes) for the row blocks in turn, then two B
  // buffers for the K stages in turn
  unsigned char* const abuf = sm;
  unsigned char* const bbuf = sm + 4 * kATile;
  // per-unit tables in K order (the even modes, then the odd modes, each
  // padded to whole stages): mode shift, phi_j (0 on padding), mode (-1)
  float* sigk = reinterpret_cast<float*>(sm + 2 * kStage);
  float* phik = sigk + kMaxKE;
  int32_t* modek = reinterpret_cast<int32_t*>(phik + kMaxKE);
  Pipe pp;
  pp.init(reinterpret_cast<unsigned char*>(modek + kMaxKE), kColsEnds);
  const uint32_t tmem = *pp.tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & (kRows - 1), half = tid >> 7;  // A row and which 32 of its 64 K
  const uint32_t idesc = idesc_bf16(128, SB);
  const int32_t L = nd.L;
  const int64_t nsb = (S + SB - 1) / SB;
  const int32_t nrb = (L + kRows - 1) / kRows;
  const int32_t ngr = (nrb + kEndsRB - 1) / kEndsRB;  // groups of kEndsRB row blocks
  const int64_t units = (int64_t)n_edges * nsb * ngr;
  // B tile item of this thread: sample bn, K chunk bc (SB x 8 <= 256 items)
  const bool bitem = tid < SB * 8;
  const int bn = tid % SB, bc = tid / SB;

  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int32_t gr = (int32_t)(u % ngr);
    const int64_t rest = u / ngr;
    const int64_t s0 = (rest % nsb) * SB;
    const int32_t e = edges[rest / nsb];
    const int32_t m = g.nel[e] - 1;
    if (m < 1) continue;
    const int32_t rb0 = gr * kEndsRB;
    const int nrbe = nrb - rb0 < kEndsRB ? nrb - rb0 : kEndsRB;  // row blocks of this unit
    const int kv = (int)(S - s0 < SB ? S - s0 : SB);
    const int64_t off = g.ioff[e];
    const float h2f = (float)(g.he[e] * g.he[e]);
    const int32_t n_even = (m + 1) / 2, n_odd = m / 2;  // modes j = 2i and j = 2i + 1
    const int ks_e = (n_even + kK - 1) / kK, ks_o = (n_odd + kK - 1) / kK;
    const int nk = ks_e + ks_o;
    const float scale = sqrtf(2.f / (float)(m + 1));
    for (int32_t p = tid; p < nk * kK; p += kT) {
      const int t = p / kK, k = p - t * kK;
      const int32_t i = (t < ks_e ? t : t - ks_e) * kK + k;
      const int32_t j = t < ks_e ? (i < n_even ? 2 * i : -1) : (i < n_odd ? 2 * i + 1 : -1);
      sigk[p] = j >= 0 ? mode_shift(j, m) : 0.f;
      phik[p] = j >= 0 ? scale * sinpif((float)(j + 1) / (float)(m + 1)) : 0.f;
      modek[p] = j;
    }
    __syncthreads();
    const float* bcol = bhat + off * S + s0 + bn;
    const bool bok = bitem && bn < kv;
    float xb[8];
    auto load_b = [&](int t, float (&x)[8]) {
      const int32_t* mk = modek + t * kK + bc * 8;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int32_t j = bok ? mk[r] : -1;
        x[r] = j >= 0 ? __ldg(bcol + (int64_t)j * S) : 0.f;
      }
    };
    load_b(0, xb);
    int last = 0;
    for (int t = 0; t < nk && !pp.failed; ++t) {
      float xn[8];
      if (t + 1 < nk) load_b(t + 1, xn);
      unsigned char* b_hi = bbuf + (t & 1) * 2 * kBPlane;
      unsigned char* b_lo = b_hi + kBPlane;
      const float* sg = sigk + t * kK + half * 32;
      for (int rb = 0; rb < nrbe; ++rb) {
        // sub-stage (t, rb) in A buffer st; acquiring it (its MMAs of two
        // sub-stages ago are done) also frees the B buffer of stage t - 2
        const int st = (t * nrbe + rb) & 1;
        last = st;
        if (!pp.acquire(st)) break;
        unsigned char* a_hi = abuf + st * 2 * kATile;
        unsigned char* a_lo = a_hi + kATile;
        if (rb == 0 && bitem) {
          const float* pk = phik + t * kK + bc * 8;
          float x[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) x[r] = pk[r] * xb[r];
          store_b_row(b_hi, b_lo, bn, bc, x);
        }
        // rows past the last node are left as they are: a GEMM row depends on
        // its own A row only, and the epilogue stores none of them
        const int32_t l = (rb0 + rb) * kRows + row;
        if (l < L) {
          const float dl = nd.shift[l] * h2f;
          const float ep = kCons ? 1.f - dl * (1.f / 6.f) : 1.f;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float4 s4a = *reinterpret_cast<const float4*>(sg + 8 * c);
            const float4 s4b = *reinterpret_cast<const float4*>(sg + 8 * c + 4);
            const float sv[8] = {s4a.x, s4a.y, s4a.z, s4a.w, s4b.x, s4b.y, s4b.z, s4b.w};
            float x[8];
#pragma unroll
            for (int r = 0; r < 8; ++r)
              x[r] = kCons ? ep * rcp_approx(fmaf(sv[r], ep, dl)) : rcp_approx(sv[r] + dl);
            store_a_row(a_hi, a_lo, row, 4 * half + c, x);
          }
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
          // odd modes from stage ks_e on, into each row block's second accumulator
          issue_stage(tmem, (uint32_t)((2 * rb + (t >= ks_e ? 1 : 0)) * SB), a_hi, a_lo, b_hi,
                      b_lo, idesc, t != 0 && t != ks_e);
          commit(&pp.mbar[st]);
        }
        pp.bump(st);
      }
      if (t + 1 < nk) {
#pragma unroll
        for (int r = 0; r < 8; ++r) xb[r] = xn[r];
      }
    }
    if (pp.failed || !pp.drain(last)) break;
    // epilogue: warp w reads lanes 32 (w % 4) .. + 31, sample half w / 4, of
    // both accumulators of each row block
    const int q4 = warp & 3, hs = warp >> 2;
    const uint32_t lanes = (uint32_t)(32 * q4) << 16;
    const int hsb = SB / 2;
    const int64_t dv = (int64_t)g.ev[e] - g.eu[e];
    for (int rb = 0; rb < nrbe; ++rb) {
      const int32_t lr = (rb0 + rb) * kRows + 32 * q4 + lane;
      const uint32_t c0 = (uint32_t)(2 * rb * SB);
      for (int cb = hs * hsb; cb < (hs + 1) * hsb; cb += 8) {
        float o[8], v[8];
        tmem_ld8(tmem + lanes + c0 + (uint32_t)cb, o);
        if (ks_o > 0) {
          tmem_ld8(tmem + lanes + c0 + (uint32_t)(SB + cb), v);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = 0.f;
        }
        if (lr < L && ends) {
          // per-edge buffer [e][end][s][l]: lanes write consecutive nodes
          float* pe = ends + ((int64_t)e * 2 * S + s0 + cb) * L + lr;
          const int64_t side = S * (int64_t)L;
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (cb + i < kv) {
              pe[(int64_t)i * L] = o[i] + v[i];
              pe[(int64_t)i * L + side] = o[i] - v[i];
            }
        } else if (lr < L) {
          double* pa = gvec + ((int64_t)lr * S + s0 + cb) * g.nv + g.eu[e];
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (cb + i < kv) {
              atomicAdd(pa, (double)(o[i] + v[i]));
              atomicAdd(pa + dv, (double)(o[i] - v[i]));
              pa += g.nv;
            }
        }
      }
    }
    fence_before();
    __syncthreads();  // accumulators and tables read before the next unit
    fence_after();
  }
  pp.finish(status);
}

// g(l, s, v) = b_v(s) + sum over the spectral edges at v of that end's value,
// from the per-edge buffer [e][end][s][l] and the sample-minor noise b. A CTA
// takes 32 vertices x 32 nodes of one sample: warp w gathers vertices
// 4w .. 4w + 3 with the lanes on consecutive nodes, and after a transpose in
// shared memory writes 32 consecutive vertices per node (FP32 sums over the
// incidences, added to b_v in FP64). Each vertex's first four sine-basis
// incidences come from one record (g.spec_inc), so the end values of all four
// vertices of a warp are requested together; the rare further incidences walk
// the incidence list.
__global__ void __launch_bounds__(256)
    ends_gather_kernel(DevGraph g, int32_t L, int64_t S, const float* __restrict__ ends,
                       const float* __restrict__ b, double* __restrict__ gvec) {
  __shared__ float tile[32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t nvt = (g.nv + 31) / 32, nlt = (L + 31) / 32;
  const int64_t tiles = (int64_t)nvt * nlt * S;
  const int64_t SL = S * (int64_t)L;  // from one (edge, end) to the next in ends
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int32_t vt = (int32_t)(t % nvt);
    const int64_t r2 = t / nvt;
    const int32_t l0 = (int32_t)(r2 % nlt) * 32;
    const int64_t s = r2 / nlt;
    const int32_t v0 = vt * 32;
    const int32_t l = l0 + lane;
    const float* __restrict__ es = ends + s * L + l;  // + (2 e + end) SL
    int4 rec[4];
    int32_t cnt[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int32_t v = v0 + 4 * warp + q;
      const bool ok = v < g.nv && l < L;
      rec[q] = ok ? __ldg(g.spec_inc + v) : make_int4(-1, -1, -1, -1);
      cnt[q] = ok ? __ldg(g.spec_cnt + v) : 0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int4 r = rec[q];
      float acc = 0.f;
      if (r.x >= 0) acc += __ldg(es + r.x * SL);
      if (r.y >= 0) acc += __ldg(es + r.y * SL);
      if (r.z >= 0) acc += __ldg(es + r.z * SL);
      if (r.w >= 0) acc += __ldg(es + r.w * SL);
      if (cnt[q] > 4) {  // the incidences after the fourth sine-basis one
        const int32_t v = v0 + 4 * warp + q;
        int32_t c = 0;
        for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
          const int32_t e = g.adj_edge[k];
          const int32_t m = g.nel[e] - 1;
          if (m < 1 || m > kMaxM) continue;  // no interior, or not a sine-basis edge
          if (c++ < 4) continue;
          const int64_t end = g.eu[e] == v ? 0 : 1;
          acc += es[(2 * (int64_t)e + end) * SL];
        }
      }
      tile[4 * warp + q][lane] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int32_t lq = l0 + 4 * warp + q, v = v0 + lane;
      if (lq < L && v < g.nv)
        gvec[((int64_t)lq * S + s) * g.nv + v] =
            (double)b[(int64_t)v * S + s] + (double)tile[lane][4 * warp + q];
    }
    __syncthreads();
  }
}

// The same sums in FP32 straight into the batched vertex PCG's layout
// g32[l][s / 8][v][s % 8] (the end values and the noise are FP32, so g carries
// their rounding already; samples past S are written as 0). A CTA takes 32
// vertices x 32 nodes x 8 samples: warp w gathers vertices 4w .. 4w + 3 with
// the lanes on consecutive nodes, and after a transpose in shared memory each
// node's 32 x 8 block is one contiguous kilobyte.
__global__ void __launch_bounds__(256)
    ends_gather32_kernel(DevGraph g, int32_t L, int64_t S, const float* __restrict__ ends,
                         const float* __restrict__ b, float* __restrict__ g32) {
  constexpr int kRow = 257;  // 32 vertices x 8 samples per node, padded
  __shared__ float tile[32 * kRow];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t nvt = (g.nv + 31) / 32, nlt = (L + 31) / 32;
  const int64_t nsg = (S + 7) / 8;
  const int64_t tiles = (int64_t)nvt * nlt * nsg;
  const int64_t SL = S * (int64_t)L;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int32_t vt = (int32_t)(t % nvt);
    const int64_t r2 = t / nvt;
    const int32_t l0 = (int32_t)(r2 % nlt) * 32;
    const int64_t sg = r2 / nlt;
    const int32_t v0 = vt * 32;
    const int32_t l = l0 + lane;
    int4 rec[4];
    int32_t cnt[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int32_t v = v0 + 4 * warp + q;
      const bool ok = v < g.nv && l < L;
      rec[q] = ok ? __ldg(g.spec_inc + v) : make_int4(-1, -1, -1, -1);
      cnt[q] = ok ? __ldg(g.spec_cnt + v) : 0;
    }
#pragma unroll 2
    for (int j = 0; j < 8; ++j) {
      const int64_t s = sg * 8 + j;
      const bool sok = s < S;
      const float* __restrict__ es = ends + (sok ? s : 0) * L + l;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int4 r = rec[q];
        float acc = 0.f;
        if (sok) {
          if (r.x >= 0) acc += __ldg(es + r.x * SL);
          if (r.y >= 0) acc += __ldg(es + r.y * SL);
          if (r.z >= 0) acc += __ldg(es + r.z * SL);
          if (r.w >= 0) acc += __ldg(es + r.w * SL);
          if (cnt[q] > 4) {  // the incidences after the fourth sine-basis one
            const int32_t v = v0 + 4 * warp + q;
            int32_t c = 0;
            for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
              const int32_t e = g.adj_edge[k];
              const int32_t m = g.nel[e] - 1;
              if (m < 1 || m > kMaxM) continue;
              if (c++ < 4) continue;
              const int64_t end = g.eu[e] == v ? 0 : 1;
              acc += es[(2 * (int64_t)e + end) * SL];
            }
          }
        }
        tile[lane * kRow + (4 * warp + q) * 8 + j] = acc;
      }
    }
    __syncthreads();
    // thread t: vertex v0 + t / 8, sample 8 sg + t % 8 of every node
    const int32_t v = v0 + (int32_t)(threadIdx.x >> 3);
    const int64_t s = sg * 8 + (threadIdx.x & 7);
    const float bv = (v < g.nv && s < S) ? b[(int64_t)v * S + s] : 0.f;
    for (int i = 0; i < 32; ++i) {
      const int32_t li = l0 + i;
      if (li >= L) break;
      if (v < g.nv)
        g32[(((int64_t)li * nsg + sg) * g.nv + v) * 8 + (threadIdx.x & 7)] =
            s < S ? bv + tile[i * kRow + threadIdx.x] : 0.f;
    }
    __syncthreads();
  }
}

// -------------------------------------------------------------- coefficients

template <bool kCons>
__global__ void __launch_bounds__(kT, 2)
    spec_coef_umma_kernel(DevGraph g, DevNodes nd, int64_t S, const int32_t* __restrict__ edges,
                          int32_t n_edges, float* __restrict__ bhat, const float* __restrict__ xw,
                          int32_t SB, PcgStatus* __restrict__ status) {
  extern __shared__ unsigned char sc_raw[];
  unsigned char* sm = align1024(sc_raw);
  const int32_t L = nd.L;
  const int nk = (L + kK - 1) / kK;
  const int LK = nk * kK;  // K positions: the nodes, padded to whole stages
  // two A buffers (hi and lo planes) for the row blocks in turn, then two B
  // buffers for the K stages in turn
  unsigned char* const abuf = sm;
  unsigned char* const bbuf = sm + 4 * kATile;
  float* bht = reinterpret_cast<float*>(sm + 2 * kStage);  // [kRows][SB] one row block's bh
  // per-unit node tables: delta_l (1 on padding), eps_l (1), sc_l (0); the
  // mode shift of each row of each row block; the partial D_j of each thread
  float* dls = bht + kRows * kMaxSB;
  float* eps = dls + LK;
  float* scs = eps + LK;
  float* sigr = scs + LK;             // [kMaxRB][kRows]
  float* dsum = sigr + kMaxRB * kRows;  // [kMaxRB][kT]
  Pipe pp;
  pp.init(reinterpret_cast<unsigned char*>(dsum + kMaxRB * kT), kColsCoef);
  const uint32_t tmem = *pp.tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & (kRows - 1), half = tid >> 7;
  const uint32_t idesc = idesc_bf16(128, SB);
  const int64_t nsb = (S + SB - 1) / SB;
  const int64_t units = (int64_t)n_edges * nsb * 2;
  const bool bitem = tid < SB * 8;
  const int bn = tid % SB, bc = tid / SB;
  const int64_t xstride = (int64_t)g.nv * S;  // from node l to node l + 1 in xw
  const bool async_bh = (S & 3) == 0;         // 16-byte row chunks

  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int par = (int)(u & 1);  // 0: even modes (xa + xb), 1: odd modes (xa - xb)
    const int64_t rest = u >> 1;
    const int64_t s0 = (rest % nsb) * SB;
    const int32_t e = edges[rest / nsb];
    const int32_t m = g.nel[e] - 1;
    const int32_t npar = par ? m / 2 : (m + 1) / 2;  // modes of this parity
    if (m < 1 || npar < 1) continue;
    const int nrbe = (npar + kRows - 1) / kRows;  // row blocks of 128 modes (<= kMaxRB)
    const int kv = (int)(S - s0 < SB ? S - s0 : SB);
    const int64_t off = g.ioff[e];
    const double h = g.he[e];
    const float hf = (float)h, h2f = (float)(h * h);
    const int32_t va = g.eu[e], vb = g.ev[e];
    // mode of row r of row block rb: j = 2 (128 rb + r) + par
    // the bh rows of row block rb, fetched asynchronously and used by its epilogue
    auto fetch_bh = [&](int rb) {
      if (!async_bh) return;
      const int cpr = SB / 4;
      for (int idx = tid; idx < kRows * cpr; idx += kT) {
        const int rr = idx / cpr, c4 = idx - rr * cpr;
        const int32_t jr = 2 * (kRows * rb + rr) + par;
        const int valid = jr < m ? (kv - 4 * c4 > 4 ? 4 : (kv - 4 * c4 > 0 ? kv - 4 * c4 : 0)) : 0;
        const float* src = bhat + (off + (jr < m ? jr : 0)) * S + s0 + (valid > 0 ? 4 * c4 : 0);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                         smem_u32(bht + rr * SB + 4 * c4)),
                     "l"(src), "r"(valid * 4)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    fetch_bh(0);
    for (int32_t p = tid; p < LK; p += kT) {
      const bool ok = p < L;
      const float d = ok ? nd.shift[p] * h2f : 1.f;
      dls[p] = d;
      eps[p] = (kCons && ok) ? 1.f - d * (1.f / 6.f) : 1.f;
      scs[p] = ok ? nd.wgam[p] * hf : 0.f;
    }
    for (int rb = 0; rb < nrbe; ++rb) {
      if (tid < kRows) {
        const int32_t j = 2 * (kRows * rb + tid) + par;
        sigr[rb * kRows + tid] = j < m ? mode_shift(j, m) : 0.f;
      }
      dsum[rb * kT + tid] = 0.f;
    }
    __syncthreads();
    const float sgn = par ? -1.f : 1.f;
    const bool bok = bitem && bn < kv;
    const float* pxa = xw + (int64_t)va * S + s0 + bn;
    const float* pxb = xw + (int64_t)vb * S + s0 + bn;
    float xa[8], xc[8];
    auto load_b = [&](int t, float (&a)[8], float (&c2)[8]) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int32_t l = t * kK + bc * 8 + r;
        const bool ok = bok && l < L;
        a[r] = ok ? __ldg(pxa + l * xstride) : 0.f;
        c2[r] = ok ? __ldg(pxb + l * xstride) : 0.f;
      }
    };
    load_b(0, xa, xc);
    int last = 0;
    for (int t = 0; t < nk && !pp.failed; ++t) {
      float na[8], nc[8];
      if (t + 1 < nk) load_b(t + 1, na, nc);
      unsigned char* b_hi = bbuf + (t & 1) * 2 * kBPlane;
      unsigned char* b_lo = b_hi + kBPlane;
      const int k0 = t * kK + half * 32;
      for (int rb = 0; rb < nrbe; ++rb) {
        // sub-stage (t, rb) in A buffer st; acquiring it (its MMAs of two
        // sub-stages ago are done) also frees the B buffer of stage t - 2
        const int st = (t * nrbe + rb) & 1;
        last = st;
        if (!pp.acquire(st)) break;
        unsigned char* a_hi = abuf + st * 2 * kATile;
        unsigned char* a_lo = a_hi + kATile;
        if (rb == 0 && bitem) {
          float xx[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const float ep = kCons ? eps[t * kK + bc * 8 + r] : 1.f;
            xx[r] = ep * fmaf(sgn, xc[r], xa[r]);
          }
          store_b_row(b_hi, b_lo, bn, bc, xx);
        }
        // rows of modes past m are left as they are (their rows of the
        // accumulator are never stored)
        const int32_t j = 2 * (kRows * rb + row) + par;
        if (j < m) {
          const float sg = sigr[rb * kRows + row];
          float D = 0.f;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float4 d4a = *reinterpret_cast<const float4*>(dls + k0 + 8 * c);
            const float4 d4b = *reinterpret_cast<const float4*>(dls + k0 + 8 * c + 4);
            const float4 s4a = *reinterpret_cast<const float4*>(scs + k0 + 8 * c);
            const float4 s4b = *reinterpret_cast<const float4*>(scs + k0 + 8 * c + 4);
            const float dv[8] = {d4a.x, d4a.y, d4a.z, d4a.w, d4b.x, d4b.y, d4b.z, d4b.w};
            const float sv[8] = {s4a.x, s4a.y, s4a.z, s4a.w, s4b.x, s4b.y, s4b.z, s4b.w};
            float ev[8] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
            if (kCons) {
              const float4 e4a = *reinterpret_cast<const float4*>(eps + k0 + 8 * c);
              const float4 e4b = *reinterpret_cast<const float4*>(eps + k0 + 8 * c + 4);
              ev[0] = e4a.x, ev[1] = e4a.y, ev[2] = e4a.z, ev[3] = e4a.w;
              ev[4] = e4b.x, ev[5] = e4b.y, ev[6] = e4b.z, ev[7] = e4b.w;
            }
            float x[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              const float a = rcp_approx(kCons ? fmaf(sg, ev[r], dv[r]) : sg + dv[r]);
              D = fmaf(sv[r], a, D);
              x[r] = a;
            }
            store_a_row(a_hi, a_lo, row, 4 * half + c, x);
          }
          dsum[rb * kT + tid] += D;
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
          issue_stage(tmem, (uint32_t)(rb * SB), a_hi, a_lo, b_hi, b_lo, idesc, t != 0);
          commit(&pp.mbar[st]);
        }
        pp.bump(st);
      }
      if (t + 1 < nk) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          xa[r] = na[r];
          xc[r] = nc[r];
        }
      }
    }
    if (pp.failed || !pp.drain(last)) break;
    // epilogue of each row block, two passes through shared memory (the A
    // buffers are free):
    // (1) warp w reads lanes 32 (w % 4) .. + 31, sample half w / 4, of the row
    //     block's accumulator into a row-major tile (SB + 1 floats a row)
    float* ct = reinterpret_cast<float*>(sm);
    float* rowd = ct + kRows * (SB + 1);  // D_j of each row
    float* rowp = rowd + kRows;           // phi_j of each row
    const int q4 = warp & 3, hs = warp >> 2;
    for (int rb = 0; rb < nrbe; ++rb) {
      {
        const int rr = 32 * q4 + lane;
        const uint32_t lanes = (uint32_t)(32 * q4) << 16;
        const int hsb = SB / 2;
        for (int cb = hs * hsb; cb < (hs + 1) * hsb; cb += 8) {
          float cv[8];
          tmem_ld8(tmem + lanes + (uint32_t)(rb * SB + cb), cv);
#pragma unroll
          for (int i = 0; i < 8; ++i) ct[rr * (SB + 1) + cb + i] = cv[i];
        }
        if (hs == 0) {
          const int32_t jr = 2 * (kRows * rb + rr) + par;
          rowd[rr] = dsum[rb * kT + rr] + dsum[rb * kT + kRows + rr];
          rowp[rr] = sqrtf(2.f / (float)(m + 1)) * sinpif((float)(jr + 1) / (float)(m + 1));
        }
      }
      if (async_bh) asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      // (2) c_j = D_j bh_j + phi_j C_j over whole rows: consecutive threads take
      //     consecutive samples of one mode, so every store is coalesced
#pragma unroll 4
      for (int idx = tid; idx < kRows * SB; idx += kT) {
        const int rr = idx / SB, sc = idx - rr * SB;
        const int32_t jr = 2 * (kRows * rb + rr) + par;
        if (jr < m && sc < kv) {
          float* o = bhat + (off + jr) * S + s0 + sc;
          const float bh = async_bh ? bht[rr * SB + sc] : *o;
          *o = fmaf(rowd[rr], bh, rowp[rr] * ct[rr * (SB + 1) + sc]);
        }
      }
      __syncthreads();  // the tile and bh rows read: the next row block's may land
      if (rb + 1 < nrbe) fetch_bh(rb + 1);
    }
    fence_before();
    __syncthreads();  // accumulators, tables and shared tiles read before the next unit
    fence_after();
  }
  pp.finish(status);
}

size_t ends_smem() { return 1024 + 2 * (size_t)kStage + 3 * (size_t)kMaxKE * 4 + 64; }
size_t coef_smem(int32_t L) {
  const size_t lk = (size_t)(L + kK - 1) / kK * kK;
  return 1024 + 2 * (size_t)kStage + kBhTile +
         (3 * lk + (size_t)kMaxRB * (kRows + kT)) * sizeof(float) + 64;
}

}  // namespace

int32_t spec_umma_sample_block(int64_t S) {
  if (S < 1) return 0;
  const int64_t r = (S + 15) / 16 * 16;
  return (int32_t)(r < kMaxSB ? r : kMaxSB);
}

bool spec_umma_fits(int32_t L) {
  return L >= 1 && ends_smem() <= kSmemLimit && coef_smem(L) <= kSmemLimit;
}

int launch_spec_ends_umma(const DevGraph& g, const DevNodes& nd, int64_t S,
                          const int32_t* bin_edges, const int32_t* bin_count, int n_bins,
                          const float* bhat, double* gvec, float* ends, const float* b,
                          bool consistent, PcgStatus* status, int n_sm, cudaStream_t st,
                          float* g32) {
  int32_t n = 0;
  for (int i = 0; i < n_bins; ++i) n += bin_count[i];
  if (n <= 0) return 0;
  const int32_t SB = spec_umma_sample_block(S);
  const size_t smem = ends_smem();
  auto kern = consistent ? spec_ends_umma_kernel<true> : spec_ends_umma_kernel<false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t nrb = (nd.L + kRows - 1) / kRows;
  const int64_t units = (int64_t)n * ((S + SB - 1) / SB) * ((nrb + kEndsRB - 1) / kEndsRB);
  const int64_t cap = 2 * (int64_t)n_sm;  // two CTAs per SM
  kern<<<(int)(units < cap ? units : cap), kT, smem, st>>>(g, nd, S, bin_edges, n, bhat, gvec,
                                                           ends, SB, status);
  if (!ends) return 1;
  const int64_t gcap = (int64_t)n_sm * 8;
  if (g32) {
    const int64_t tiles = (int64_t)((g.nv + 31) / 32) * ((nd.L + 31) / 32) * ((S + 7) / 8);
    ends_gather32_kernel<<<(int)(tiles < gcap ? tiles : gcap), 256, 0, st>>>(g, nd.L, S, ends, b,
                                                                             g32);
    return 2;
  }
  const int64_t tiles = (int64_t)((g.nv + 31) / 32) * ((nd.L + 31) / 32) * S;
  ends_gather_kernel<<<(int)(tiles < gcap ? tiles : gcap), 256, 0, st>>>(g, nd.L, S, ends, b,
                                                                         gvec);
  return 2;
}

int launch_spec_coef_umma(const DevGraph& g, const DevNodes& nd, int64_t S,
                          const int32_t* bin_edges, const int32_t* bin_count, int n_bins,
                          float* bhat, const float* xw, bool consistent, PcgStatus* status,
                          int n_sm, cudaStream_t st) {
  int32_t n = 0;
  for (int i = 0; i < n_bins; ++i) n += bin_count[i];
  if (n <= 0) return 0;
  const int32_t SB = spec_umma_sample_block(S);
  const size_t smem = coef_smem(nd.L);
  auto kern = consistent ? spec_coef_umma_kernel<true> : spec_coef_umma_kernel<false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // one unit per (edge, sample block, parity), all its row blocks of modes
  const int64_t units = (int64_t)n * ((S + SB - 1) / SB) * 2;
  const int64_t cap = 2 * (int64_t)n_sm;
  kern<<<(int)(units < cap ? units : cap), kT, smem, st>>>(g, nd, S, bin_edges, n, bhat, xw, SB,
                                                           status);
  return 1;
}

}  // namespace grf
