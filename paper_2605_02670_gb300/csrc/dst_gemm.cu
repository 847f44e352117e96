// The sine transforms of the spectral edge-interior path on the 5th-generation
// tensor cores (tcgen05.mma, accumulator in tensor memory).
//
// On an edge with m interior nodes the transform pair of the sine-basis
// solves (Sec. 3 Phases 3 and 5 through the exact change of basis of the
// uniform lumped edge mesh: T_l = Phi diag(mu_l) Phi for every node l) is
//   forward  bh = Phi b_I   (condensation),   inverse  U_I = Phi c   (recovery),
// with the same symmetric Phi_ji = sqrt(2/(m+1)) sin(pi (j+1)(i+1)/(m+1)) for
// every edge of that length. Edges are grouped by m, so each group's
// transforms are one dense product Phi_m [m x m] by [m x (edges x samples)]:
// Phi_m is built once per graph and every column of the group shares it.
//
// Precision: FP32 operands as split BF16 pairs a = a_hi + a_lo (a_lo the BF16
// rounding of a - a_hi; |a - a_hi - a_lo| <= 2^-17 |a|), products formed as
// a_hi b_hi + a_hi b_lo + a_lo b_hi with FP32 accumulation in tensor memory
// (relative error about 2^-16 per product), inside the FP32 tolerance of the
// mixed-precision path.
//
// One CTA per SM; a work item is a 128-row block of Phi_m (modes, or output
// nodes) times a 256-column block (256 / Sp edges of Sp padded samples). K runs
// in stages of 64 (one 128-byte swizzle row of BF16), double-buffered in
// shared memory: all threads load and split stage k+1 while the tensor core
// runs the 12 MMAs (4 K-steps x 3 products) of stage k, issued by one thread
// and signalled to an mbarrier by tcgen05.commit. The accumulator
// (128 lanes x 256 FP32 columns) is read back with tcgen05.ld. Every mbarrier
// wait is bounded: on a timeout the CTA raises the error flag, waits (bounded)
// for its MMAs, frees its tensor memory and stops.
#include "grf_internal.h"

namespace grf {
namespace {

constexpr int kGT = 256;   // threads per CTA
constexpr int kBM = 128;   // rows of a tile (UMMA M)
constexpr int kBN = 256;   // columns of a tile (UMMA N)
constexpr int kBK = 64;    // K per stage
constexpr int kStages = 2;
constexpr uint32_t kATile = kBM * kBK * 2;                 // 16 KB (BF16)
constexpr uint32_t kBTile = kBN * kBK * 2;                 // 32 KB
constexpr uint32_t kStageBytes = 2 * kATile + 2 * kBTile;  // hi and lo planes
constexpr uint32_t kSmemBytes = kStages * kStageBytes + 1024 + 128;
constexpr uint32_t kTmemCols = 256;
// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major,
// N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
constexpr unsigned long long kWaitNs = 2000000000ull;  // give up a wait after 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128
// bytes, 8-row groups 1024 bytes apart (the tile base is 1024-byte aligned).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Waits for the completion of the phase with the given parity; false once
// kWaitNs have passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const unsigned long long t0 = now_ns();
  for (long long i = 0;; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 255) == 255 && now_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half)
  return *reinterpret_cast<const uint32_t*>(&h);
}

// hi/lo BF16 split of 8 values into two 16-byte chunks
__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
  float h[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const __nv_bfloat16 b = __float2bfloat16_rn(x[i]);
    h[i] = __bfloat162float(b);
    l[i] = x[i] - h[i];
  }
  hi = make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]),
                  pack_bf16(h[6], h[7]));
  lo = make_uint4(pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]), pack_bf16(l[4], l[5]),
                  pack_bf16(l[6], l[7]));
}

// byte offset of 16-byte chunk c of row r in a 128-byte-swizzled tile
__device__ __forceinline__ uint32_t swz(int r, int c) {
  return (uint32_t)r * 128u + (uint32_t)((c ^ (r & 7)) << 4);
}

// Phi_m hi/lo planes: [mp][kp] row-major, zero outside j, i < m.
__global__ void phi_planes_kernel(const DstGroup* __restrict__ groups, int32_t n_groups,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  for (int32_t gi = blockIdx.y; gi < n_groups; gi += gridDim.y) {
    const DstGroup G = groups[gi];
    const int64_t total = (int64_t)G.mp * G.kp;
    const double sc = sqrt(2.0 / (double)(G.m + 1));
    const int64_t P = 2 * (int64_t)(G.m + 1);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
      const int64_t j = t / G.kp, i = t - j * G.kp;
      float vh = 0.f, vl = 0.f;
      if (j < G.m && i < G.m) {
        const int64_t q = ((j + 1) * (i + 1)) % P;  // exact argument reduction
        const double v = sc * sinpi((double)q / (double)(G.m + 1));
        const __nv_bfloat16 h = __double2bfloat16(v);
        vh = __bfloat162float(h);
        vl = (float)(v - (double)vh);
      }
      hi[G.phi_off + t] = __float2bfloat16_rn(vh);
      lo[G.phi_off + t] = __float2bfloat16_rn(vl);
    }
  }
}

// kInv = false: bhat[(ioff_e + j) S + s] = sum_i Phi_ji b[(nv + ioff_e + i) S + s]
// kInv = true:  out[s n + nv + ioff_e + i] = sum_j Phi_ij c[(ioff_e + j) S + s]
template <bool kInv, typename OutT>
__global__ void __launch_bounds__(kGT, 1)
    dst_gemm_kernel(DevGraph g, const DstItem* __restrict__ items, int32_t n_items,
                    const int32_t* __restrict__ edges, const __nv_bfloat16* __restrict__ phi_hi,
                    const __nv_bfloat16* __restrict__ phi_lo, int64_t S, int32_t sp,
                    const float* __restrict__ src, OutT* __restrict__ dst,
                    PcgStatus* __restrict__ status) {
  extern __shared__ unsigned char dg_raw[];
  const uint32_t raw = smem_u32(dg_raw);
  unsigned char* sm = dg_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kStages * kStageBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + kStages);
  int* fail_flag = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&mbar[s], 1);
    *fail_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  uint32_t uses[kStages] = {0, 0};  // commits to each stage's barrier so far
  bool failed = false;

  const int ept = kBN / sp;  // edges per tile
  for (int32_t item = blockIdx.x; item < n_items && !failed; item += gridDim.x) {
    const DstItem it = items[item];
    // this thread's B column: edge slot tid / sp, sample tid % sp
    const int et = tid / sp, s = tid % sp;
    const bool col_ok = et < it.ne && s < S;
    const int32_t ecol = col_ok ? edges[it.e0 + et] : 0;
    const int64_t row0 = col_ok ? (kInv ? g.ioff[ecol] : (int64_t)g.nv + g.ioff[ecol]) : 0;
    const float* colp = src + row0 * S + s;
    const __nv_bfloat16* ah = phi_hi + it.phi_off + (int64_t)it.mt * kBM * it.kp;
    const __nv_bfloat16* al = phi_lo + it.phi_off + (int64_t)it.mt * kBM * it.kp;
    const int nk = it.kp / kBK;
    int last = 0;
    // B values of the next stage are loaded into registers one stage ahead,
    // so their latency overlaps the previous stage's MMAs and barrier wait
    float xb[8][8];
    auto load_b = [&](int kb, float (&x)[8][8]) {
#pragma unroll
      for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int k = kb * kBK + c * 8 + q;
          x[c][q] = (col_ok && k < it.m) ? __ldg(colp + (int64_t)k * S) : 0.f;
        }
    };
    load_b(0, xb);
    for (int kb = 0; kb < nk; ++kb) {
      const int st = kb & 1;
      last = st;
      float xn[8][8];
      if (kb + 1 < nk) load_b(kb + 1, xn);
      if (uses[st] > 0 && !mbar_wait(&mbar[st], (uses[st] - 1) & 1)) failed = true;
      if (__syncthreads_or(failed)) {
        failed = true;
        break;
      }
      unsigned char* A_hi = sm + st * kStageBytes;
      unsigned char* A_lo = A_hi + kATile;
      unsigned char* B_hi = A_lo + kATile;
      unsigned char* B_lo = B_hi + kBTile;
      // A: 128 rows x 8 chunks of 16 bytes per plane, copied asynchronously
#pragma unroll
      for (int u = 0; u < (kBM * 8) / kGT; ++u) {
        const int idx = tid + u * kGT;
        const int r = idx >> 3, c = idx & 7;
        const int64_t go = (int64_t)r * it.kp + kb * kBK + c * 8;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(A_hi + swz(r, c))),
                     "l"(ah + go)
                     : "memory");
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(A_lo + swz(r, c))),
                     "l"(al + go)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      // B: column tid, 64 K values in 8 chunks of 8, split into hi/lo
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint4 hi, lo;
        split8(xb[c], hi, lo);
        *reinterpret_cast<uint4*>(B_hi + swz(tid, c)) = hi;
        *reinterpret_cast<uint4*>(B_lo + swz(tid, c)) = lo;
      }
      if (kb + 1 < nk) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
          for (int q = 0; q < 8; ++q) xb[c][q] = xn[c][q];
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      // make the generic-proxy stores visible to the tensor core
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint64_t dah = sdesc(smem_u32(A_hi)), dal = sdesc(smem_u32(A_lo));
        const uint64_t dbh = sdesc(smem_u32(B_hi)), dbl = sdesc(smem_u32(B_lo));
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
          const uint64_t o = (uint64_t)(kk * 32) >> 4;  // 16 BF16 = 32 bytes along K
          umma_bf16(tmem, dah + o, dbh + o, (kb | kk) != 0);
          umma_bf16(tmem, dah + o, dbl + o, 1u);
          umma_bf16(tmem, dal + o, dbh + o, 1u);
        }
        umma_commit(&mbar[st]);
      }
      uses[st] += 1;
    }
    if (failed) break;
    // the last commit covers every MMA of this item
    if (!mbar_wait(&mbar[last], (uses[last] - 1) & 1)) failed = true;
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    tc_fence_after();
    // epilogue: warp w reads lanes 32 (w % 4) .. + 31, columns 128 (w / 4) .. + 127
    const int q4 = warp & 3, half = warp >> 2;
    const int row = 32 * q4 + lane;
    const int32_t jrow = it.mt * kBM + row;  // mode (forward) or output node (inverse)
#pragma unroll 1
    for (int cb = 0; cb < 4; ++cb) {
      const int col0 = 128 * half + 32 * cb;
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)col0, v);
      if (jrow >= it.m) continue;
      if (!kInv && sizeof(OutT) == 4 && sp >= 32 && (S & 3) == 0) {
        // the 32 columns are 32 consecutive samples of one edge: 8 vector stores
        const int e_t = col0 / sp, sc0 = col0 % sp;
        if (e_t < it.ne && sc0 + 32 <= S) {
          const int32_t e = edges[it.e0 + e_t];
          float4* row = reinterpret_cast<float4*>(
              reinterpret_cast<float*>(dst) + (g.ioff[e] + jrow) * S + sc0);
#pragma unroll
          for (int t = 0; t < 8; ++t)
            row[t] = make_float4(v[4 * t], v[4 * t + 1], v[4 * t + 2], v[4 * t + 3]);
          continue;
        }
      }
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int n = col0 + t;
        const int e_t = n / sp, sc = n % sp;
        if (e_t >= it.ne || sc >= S) continue;
        const int32_t e = edges[it.e0 + e_t];
        if (kInv)
          dst[(int64_t)sc * g.n + g.nv + g.ioff[e] + jrow] = (OutT)v[t];
        else
          dst[(g.ioff[e] + jrow) * S + sc] = (OutT)v[t];
      }
    }
    tc_fence_before();
    __syncthreads();  // accumulator read before the next item's first MMA
    tc_fence_after();
  }
  if (failed) {
    if (tid == 0) atomicAdd(&status->device_timeout, 1);
    // let MMAs still in flight finish (bounded) before the memory is freed
    for (int s = 0; s < kStages; ++s)
      if (uses[s] > 0) mbar_wait(&mbar[s], (uses[s] - 1) & 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

}  // namespace

int32_t dst_gemm_sample_pad(int64_t S) {
  if (S < 1 || S > kBN) return 0;
  int32_t p = 8;
  while (p < S) p *= 2;
  return p;
}

int32_t dst_gemm_tile_rows() { return kBM; }
int32_t dst_gemm_tile_k() { return kBK; }
int32_t dst_gemm_tile_cols() { return kBN; }

void launch_phi_planes(const DstGroup* groups, int32_t n_groups, __nv_bfloat16* hi,
                       __nv_bfloat16* lo, cudaStream_t st) {
  if (n_groups <= 0) return;
  const int gy = n_groups < 65535 ? n_groups : 65535;
  phi_planes_kernel<<<dim3(64, gy), 256, 0, st>>>(groups, n_groups, hi, lo);
}

template <bool kInv, typename OutT>
int launch_dst_gemm(const DevGraph& g, const DstPlanDev& p, int64_t S, const float* src,
                    OutT* dst, PcgStatus* status, int n_sm, cudaStream_t st) {
  if (p.n_items <= 0) return 0;
  cudaFuncSetAttribute(dst_gemm_kernel<kInv, OutT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kSmemBytes);
  const int grid = p.n_items < n_sm ? p.n_items : n_sm;
  dst_gemm_kernel<kInv, OutT><<<grid, kGT, kSmemBytes, st>>>(
      g, p.items, p.n_items, p.edges, p.phi_hi, p.phi_lo, S, p.sp, src, dst, status);
  return 1;
}
template int launch_dst_gemm<false, float>(const DevGraph&, const DstPlanDev&, int64_t,
                                           const float*, float*, PcgStatus*, int, cudaStream_t);
template int launch_dst_gemm<true, float>(const DevGraph&, const DstPlanDev&, int64_t,
                                          const float*, float*, PcgStatus*, int, cudaStream_t);
template int launch_dst_gemm<true, double>(const DevGraph&, const DstPlanDev&, int64_t,
                                           const float*, double*, PcgStatus*, int, cudaStream_t);

}  // namespace grf
