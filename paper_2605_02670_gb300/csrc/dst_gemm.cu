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
#include "umma.cuh"

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
constexpr uint32_t kIdesc = umma::idesc_bf16(kBM, kBN);  // N = 256, M = 128

using namespace umma;

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
    tmem_alloc(tslot, kTmemCols);
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  uint32_t uses[kStages] = {0, 0};  // commits to each stage's barrier so far
  bool failed = false;

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
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        fence_after();
        const uint64_t dah = sdesc(smem_u32(A_hi)), dal = sdesc(smem_u32(A_lo));
        const uint64_t dbh = sdesc(smem_u32(B_hi)), dbl = sdesc(smem_u32(B_lo));
        mma_split_stage(tmem, dah, dal, dbh, dbl, kIdesc, kb != 0);
        commit(&mbar[st]);
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
    fence_after();
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
    fence_before();
    __syncthreads();  // accumulator read before the next item's first MMA
    fence_after();
  }
  if (failed) {
    if (tid == 0) atomicAdd(&status->device_timeout, 1);
    // let MMAs still in flight finish (bounded) before the memory is freed
    for (int s = 0; s < kStages; ++s)
      if (uses[s] > 0) mbar_wait(&mbar[s], (uses[s] - 1) & 1);
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    tmem_dealloc(tmem, kTmemCols);
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
