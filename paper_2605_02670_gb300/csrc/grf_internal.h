// Internal declarations shared by the sampler's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace grf {

// Multiprocessors of the current device, read once per device: the grid caps
// of the grid-stride launchers are multiples of it.
inline int sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n == 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 152;
    cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

// Device copy of the mesh (Sec. 3, Phase 1). Vertex ids are kept ids.
constexpr int32_t kSpecMaxM = 1024;  // interior nodes of the longest sine-basis edge

struct DevGraph {
  int32_t nv;        // kept vertices
  int32_t ne;        // edges
  int64_t ni;        // interior nodes
  int64_t n;         // DOFs = nv + ni
  int32_t max_m;     // largest interior node count of an edge
  const int32_t* eu;     // [ne] endpoint at x = 0
  const int32_t* ev;     // [ne] endpoint at x = l_e
  const int32_t* nel;    // [ne] elements n_e (>= 1)
  const double* he;      // [ne] element size h_e
  const int64_t* ioff;   // [ne + 1] interior offsets
  const int32_t* vptr;   // [nv + 1] vertex -> incidence list
  const int32_t* adj_edge;  // [2 ne] incident edge
  const int32_t* adj_nbr;   // [2 ne] vertex at the other end
  const int32_t* adj_rev;   // [2 ne] index of the same edge in the other end's list
  const double* sqrt_ml;    // [n] sqrt of the lumped mass per DOF
  // per vertex its first four incidences on sine-basis edges (1 <= m <= 1024)
  // as 2 e + end (end 0 at x = 0), -1 past them, and how many it has in all
  const int4* spec_inc;     // [nv]: edges with m <= kSpecMaxM count
  const int32_t* spec_cnt;  // [nv]
};

// A renumbering of the vertices into slots (reverse Cuthill-McKee order,
// computed once per graph) and the incidence lists in slot order. Kept apart
// from DevGraph: only the shared-memory vertex PCG uses it.
struct VertexOrder {
  const int32_t* perm;  // [nv] slot -> vertex
  const int32_t* vptr;  // [nv + 1] slot -> incidence list
  const int32_t* nbr;   // [2 ne] slot of the vertex at the other end
  const int32_t* inc;   // [2 ne] index of the same incidence in DevGraph's lists
};

// Per-call node list: A_l = alpha_l M_L + gamma_l K, weight w_l.
struct DevNodes {
  int32_t L;
  const double* alpha;
  const double* gamma;
  const double* weight;
  // FP32 per-node constants of the FP32 interior kernels (may be null):
  // shift_l = alpha_l / gamma_l + kappa^2 (delta_l = shift_l h_e^2) and
  // wgam_l = w_l / gamma_l (w_l / c_l = wgam_l h_e)
  const float* shift = nullptr;
  const float* wgam = nullptr;
};

struct PcgStatus {
  int32_t n_unconverged;
  int32_t numeric_flag;
  int32_t iters_max;
  int32_t n_fallback;  // systems whose learned preconditioner fell back to Jacobi
  int32_t device_timeout;  // tensor-core kernels whose bounded waits ran out
  int32_t pad;
  unsigned long long iters_total;
};

// ---- noise.cu
// b[j][s] (sample-minor, T = float or double) = sqrt(M_L,j) xi_{s,j};
// the seed is read from seed_dev when it is not null (graph replays); the FP32
// form scales by sqrt_ml_f (an FP32 copy of g.sqrt_ml) when it is given.
template <typename T>
void launch_noise_minor(const DevGraph& g, uint64_t seed, int64_t S, T* b, cudaStream_t st,
                        const uint64_t* seed_dev = nullptr, const float* sqrt_ml_f = nullptr);
// sample-major output: raw words (uint32) or b in double
void launch_noise_major(const DevGraph& g, uint64_t seed, int64_t S, void* out, bool raw,
                        cudaStream_t st);

// Per-(node, edge) constants of the interior sweeps in the sweep precision T:
// delta, w_l h_e / gamma_l (= w_l / c), sinh(theta), theta with
// 2 + delta = 2 cosh(theta).
template <typename T>
struct alignas(4 * sizeof(T)) SweepParams {
  T delta, sc, sh, theta;
};

// ---- schur.cu
// Per-(l, e) 2x2 Schur blocks and vertex diagonal:
//   saa[l][e], sab[l][e];  diag[l][v] = sum_{e at v} saa[l][e];
//   offv[l][k] = sab[l][adj_edge[k]] in vertex-incidence order;
//   prm[l][e] (if not null): the sweep constants above;
//   dscale[l][v] (if not null): 1 / S_vv (T = double) or 1 / sqrt(S_vv) (T = float);
//   offv_t (T = float, if not null): offv / sqrt(S_vv S_ww);
//   dpair[l][v], opair[l][k] (if not null): diag and offv as FP32 pairs
//   (hi = fl32(x), lo = fl32(x - hi)).
// Returns the number of kernels launched.
// consistent: blocks of the consistent-mass operator (no sweep constants).
template <typename T>
int launch_schur(const DevGraph& g, const DevNodes& nd, double kappa2, double* saa,
                 double* sab, double* diag, double* offv, SweepParams<T>* prm, T* dscale,
                 T* offv_t, cudaStream_t st, bool consistent = false, float2* dpair = nullptr,
                 float2* opair = nullptr);

// Neumann-Neumann preconditioner coefficients per node: pc[l][v] (diagonal) and
// pn[l][k] (incidence k), for the Jacobi-scaled system (scaled) or S itself.
template <typename T>
void launch_nn_coeffs(const DevGraph& g, int32_t L, const double* saa, const double* sab,
                      const double* diag, bool scaled, T* pc, T* pn, cudaStream_t st);

// ---- thomas.cu
// rhs (sample-minor [n][S], T) -> condensed right-hand side gvec[l][s][v] (double):
// gvec = b at the vertices plus the end values of the listed edges (edges null:
// every edge); init = false: gvec already holds b plus other edges' values and
// only the listed edges are added. Returns the number of kernels launched.
template <typename T>
int launch_condense(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S,
                    const T* b, double* gvec, cudaStream_t st, const int32_t* edges = nullptr,
                    int32_t n_edges = 0, bool init = true);
// Vertex accumulation out[s][v] = sum_l w_l x[l][s][v], and fused interior
// recovery + quadrature sum for the interior DOFs: binned register-resident
// kernels (recover.cu) for edges up to the largest bin, the sequential kernel
// for longer ones (bin_count[n_bins] of them, listed last in bin_edges; they
// need acc/yscr/rpscr, sized [n_interior][S]). bin_count is a host array.
// Returns the number of kernels launched.
// prm: sweep constants from launch_schur; xw: [L][nv][S] scratch that receives
// w_l u_v^(l) in precision T (sample-minor). xw_ready: xw already holds them
// (FP32, written by the batched PCG) and xv is not read: the vertex values are
// their sums over the nodes.
template <typename T, typename OutT>
int launch_recover(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S,
                   const T* b, const double* xv, OutT* out, const SweepParams<T>* prm, T* xw,
                   const int32_t* bin_edges, const int32_t* bin_count, int32_t n_bins,
                   double* acc, T* yscr, T* rpscr, int sg, cudaStream_t st,
                   bool xw_ready = false);
// ---- sweep.cu (FP32 interiors)
// Node-parallel sweeps: one warp per (edge, 4 samples), each lane a set of
// quadrature nodes (at most kNodeSweepMaxNL per lane, so L <= 32 kNodeSweepMaxNL).
// condense: adds the listed edges' end values into gvec (after launch_condense's
// vertex init); recover: writes the listed edges' interior DOFs of out.
// Both need the sweep constants prm of launch_schur. Return the launch count.
constexpr int kNodeSweepMaxNL = 8;
bool node_sweep_fits(int32_t L);
int launch_condense_nodes(const DevGraph& g, int32_t L, int64_t S, const float* b,
                          const SweepParams<float>* prm, const int32_t* edges, int32_t n_edges,
                          double* gvec, cudaStream_t st);
template <typename OutT>
int launch_recover_nodes(const DevGraph& g, int32_t L, int64_t S, const float* b,
                         const SweepParams<float>* prm, const float* xw, const int32_t* edges,
                         int32_t n_edges, OutT* out, cudaStream_t st);
// [S][n] double -> [n][S] T, each DOF j scaled by scale[j] (or 1 when scale is null
// and mass_scale is false; by M_L,j = sqrt_ml[j]^2 when mass_scale is true)
template <typename T>
void launch_to_minor(const DevGraph& g, int64_t S, const double* src, T* dst, bool mass_scale,
                     cudaStream_t st);

// ---- pcg.cu
// Vertex PCG for all L x S systems; x[l][s][v] (FP64) receives the solution.
// VT = double: FP64 Jacobi-PCG (dscale = 1 / D, offv_t = offv).
// VT = float: FP32 Jacobi-scaled CG inside FP64 refinement (dscale = 1 / sqrt(D),
// offv_t = scaled blocks). d, r, p, q: [L][S][nv] scratch used when a system's
// vectors do not fit in shared memory. layout: 1 one CTA per system, 2 staged
// matrix per (node, sample group) when it fits (mixed only), else layout 1;
// the sample-group Jacobi kernel stores its system in the slot order ord.
// Preconditioner: pre = kPreJacobi (pc, pn unused), kPreNeumann (pc [L][V] and
// pn [L][2E] in VT: z_v = pc_v r_v + sum_k pn_k r_nbr(k)) or kPreLearned (mixed
// only, float es = pc and N = pn per node: z = B B^T r, B = diag(es) + N);
// y: one more [L][S][nv] scratch for the learned form.
constexpr int kPreJacobi = 0, kPreNeumann = 1, kPreLearned = 2;

// ---- pcg_batch.cu
// Mixed-precision Jacobi-PCG with one CTA per (node, 8 samples) and the
// group's FP32 vectors as [nv][8] rows in global memory (graphs whose vectors
// do not fit on chip). R, PA, PB, Dv: [L][ceil(S / 8)][nv][8] floats each.
// ell: nv int4 (each vertex's first four neighbours, padded with itself),
// then nv int2 (incidence-list start, degree).
int64_t pcg_batch_padded_samples(int64_t S);
// Extra state of the batched layout's refinement, which runs in FP32-pair
// arithmetic: the FP64 blocks as pairs (launch_schur's dpair [L][V], opair
// [L][2E]) and four more vectors of the batched shape (iterate hi/lo and
// scaled right-hand side hi/lo).
struct PcgPairs {
  const float2* dp;
  const float2* op;
  float *xh, *xl, *gh, *gl;
  // true: gh already holds g in FP32 (launch_spec_ends_umma's g32) and the
  // FP64 gvec is not read
  bool g32;
  // not null: the solutions leave as the recovery's weighted values
  // xw[l][v][s] = w_l u_v^(l) (FP32, weight = the node weights w_l) instead of
  // the FP64 x
  float* xw;
  const double* weight;
  double* gn;  // [L][S] scratch for ||g|| of each system (with xw)
};
void launch_pcg_batch(const DevGraph& g, const int4* ell, int32_t L, int64_t S, const double* diag,
                      const double* offv, const float* dscale, const float* offv_t,
                      const double* gvec, double* x, float* R, float* PA, float* PB, float* Dv,
                      const PcgPairs& pp, double rtol, int32_t max_iter, int32_t* iters,
                      PcgStatus* status, cudaStream_t st);
// Whether launch_pcg<float> with pairs takes the batched layout.
bool pcg_batch_selected(const DevGraph& g, int layout, int pre);
// pairs: required by the batched layout (FP32 only), ignored otherwise.
template <typename VT>
void launch_pcg(const DevGraph& g, const VertexOrder& ord, const int4* ell, int32_t L, int64_t S,
                const double* diag, const double* offv, const VT* dscale_t, const VT* offv_t, int pre, const VT* pc, const VT* pn,
                const double* gvec, double* x, VT* d, VT* r, VT* p, VT* q, VT* y, double rtol,
                int32_t max_iter, int32_t* iters, PcgStatus* status, int layout,
                cudaStream_t st, const PcgPairs* pairs);

int recover_sample_group();

// ---- learned.cu: learned BB^T preconditioner of the scaled Schur systems.
// FP32 parameter vector layout (fixed flat order):
// W0 [8 x 64], b0, then W_i [128 x 64], b_i for i = 1..3, then ws [64], cs, u [64],
// up [64], cn.
constexpr int kFeat = 8;
constexpr int kLayers = 3;
constexpr int kOffW0 = 0;
constexpr int kOffB0 = kFeat * 64;
__host__ __device__ constexpr int layer_w_off(int i) { return kOffB0 + 64 + (i - 1) * (8192 + 64); }
constexpr int kOffWs = layer_w_off(kLayers + 1);
constexpr int kOffCs = kOffWs + 64;
constexpr int kOffU = kOffCs + 1;
constexpr int kOffUp = kOffU + 64;
constexpr int kOffCn = kOffUp + 64;
constexpr int kParams = kOffCn + 1;
constexpr int kWbf16 = 16 * 64 + 3 * 8192;  // BF16 copies: W0 padded to 16 rows, W1..W3
constexpr int kWtbf16 = 3 * 8192;           // W1..W3 transposed

// Activations of a forward pass over Lb nodes (M = Lb * V rows).
struct LpActs {
  __nv_bfloat16* X0;     // [M x 16]
  float* H[kLayers + 1]; // [M x 64]
  __nv_bfloat16* Xc[kLayers];  // [M x 128] = [h_{i-1} | m_i]
  float *s, *es, *al, *be;     // [M]
  float* n;                    // [Lb x 2E]
};
struct LpGrads {
  float *ds, *dn;        // [M], [Lb x 2E]
  float *dH, *dX;        // [M x 64], [M x 128]
  __nv_bfloat16* dA;     // [M x 64]
  float* scratch;        // [max_pair_ctas x 4 V]
  int max_pair_ctas;
};

void lp_weights_bf16(const float* P, __nv_bfloat16* wb, __nv_bfloat16* wt, cudaStream_t st);
// Returns the number of kernels launched.
int lp_forward(const DevGraph& g, int32_t Lb, const int32_t* lnode, const float* offv_t,
               const double* alpha, const double* gamma, const float* P,
               const __nv_bfloat16* wb, const LpActs& a, cudaStream_t st);
void lp_backward(const DevGraph& g, int32_t Lb, const int32_t* lnode, const float* offv_t,
                 const float* P, const __nv_bfloat16* wt, const LpActs& a, int64_t npairs,
                 const int32_t* pj, const int64_t* slot, const float* R, const float* E,
                 float inv_p, const LpGrads& b, float* G, float* loss, cudaStream_t st);
void lp_adam(float* P, float* G, float* m, float* v, float lr, int step, cudaStream_t st);
void lp_record_pairs(const DevGraph& g, int64_t nsys, int64_t S, const double* diag,
                     const double* offv, const double* gvec, double* work, double* xrec,
                     float* R, float* E, double* rinv, int32_t* count, int per_sys, int stride,
                     double rtol, int max_iter, int ctas, cudaStream_t st);

// ---- spectral.cu: edge interiors in the sine basis (FP32 sweeps only).
// shift[l], wgam[l] of DevNodes from alpha, gamma, weight (one launch).
void launch_node_consts(const DevNodes& nd, double kappa2, float* shift, float* wgam,
                        cudaStream_t st);
// Spectral bins: bin i holds edges with 1 <= m <= mmax[i] interior nodes (and
// above the previous bin's limit). Returns the number of bins.
constexpr int kSpecSG = 16;  // samples per CTA
int spec_bins(int32_t* mmax);
// bhat [n_interior][S] receives the sine transform of the interior noise rows;
// gvec [L][S][nv] gets the two end values of T_l^-1 b_I added per edge.
int launch_spec_condense(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S,
                         const float* b, const int32_t* bin_edges, const int32_t* bin_count,
                         float* bhat, double* gvec, cudaStream_t st);
// The same on the tensor cores (spectral_mma.cu): mma.sync TF32 in three terms.
int launch_spec_condense_mma(const DevGraph& g, const DevNodes& nd, int64_t S, const float* b,
                             const int32_t* bin_edges, const int32_t* bin_count, float* bhat,
                             double* gvec, cudaStream_t st);
// Interior field of the binned edges from bhat and xw = w_l u_v^(l).
template <typename OutT>
int launch_spec_recover(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S,
                        const int32_t* bin_edges, const int32_t* bin_count, const float* bhat,
                        const float* xw, OutT* out, cudaStream_t st);
// ---- spec_umma.cu: the two node contractions around the tensor-core sine
// transforms (dst_gemm.cu) on the tensor cores (tcgen05, BF16 hi/lo operands
// in three products, FP32 accumulation): the end values of every node from
// bhat (already transformed) added into gvec, and the sine-basis coefficients
// c of the recovery written over bhat (the inverse transform of c is then the
// interior field). bin_edges / bin_count: the spectral edges over n_bins bins;
// consistent: the consistent-mass operator (interior constants transformed).
// Samples run in blocks of spec_umma_sample_block(S) (a multiple of 16, at
// most 64; at most 32 for the coefficients); the shared memory of the
// coefficient kernel grows with L (spec_umma_fits). ends: a scratch of
// 2 E S L floats for the end values per edge, then gathered over the vertices'
// incidences into gvec = b_v + (end values), b the sample-minor noise: this
// initialises gvec (null ends: FP64 atomics into an initialised gvec). With
// g32 (and ends) the sums go in FP32 to g32 in the batched PCG's layout
// [L][ceil(S / 8)][nv][8] instead, and gvec is not touched.
int32_t spec_umma_sample_block(int64_t S);
bool spec_umma_fits(int32_t L);
int launch_spec_ends_umma(const DevGraph& g, const DevNodes& nd, int64_t S,
                          const int32_t* bin_edges, const int32_t* bin_count, int n_bins,
                          const float* bhat, double* gvec, float* ends, const float* b,
                          bool consistent, PcgStatus* status, int n_sm, cudaStream_t st,
                          float* g32 = nullptr);
int launch_spec_coef_umma(const DevGraph& g, const DevNodes& nd, int64_t S,
                          const int32_t* bin_edges, const int32_t* bin_count, int n_bins,
                          float* bhat, const float* xw, bool consistent, PcgStatus* status,
                          int n_sm, cudaStream_t st);

// ---- consistent.cu: white noise of the consistent mass, W = R xi with the
// Cholesky order interiors (edge by edge) then vertices. On entry b [n][S]
// holds unit-mass standard normals; on return W. wv: [nv][S] scratch;
// (rp, rc, rv): the lower factor of the vertex Schur complement of the mass
// (CSR, kept-vertex order). Returns the launch count.
int launch_cons_noise(const DevGraph& g, int64_t S, float* b, float* wv, const int64_t* rp,
                      const int32_t* rc, const float* rv, int n_sm, cudaStream_t st);
// out[s][j] = b[j][s] (FP32 sample-minor to FP64 sample-major)
void launch_minor_to_major(int64_t n, int64_t S, const float* b, double* out, cudaStream_t st);

// ---- dst_gemm.cu: sine transforms of edges grouped by interior-node count m,
// as BF16-split products on the tcgen05 tensor cores.
// A group: edges with m interior nodes; Phi_m's hi and lo planes start at
// phi_off ([mp][kp], mp, kp rounded up to the tile rows and K).
struct DstGroup {
  int64_t phi_off;
  int32_t m, mp, kp, pad;
};
// A work item: rows [128 mt, 128 mt + 128) of Phi_m times ne <= 256 / sp edges
// (edges[e0 .. e0 + ne)).
struct DstItem {
  int64_t phi_off;
  int32_t m, kp, e0, ne, mt, pad;
};
struct DstPlanDev {
  const __nv_bfloat16* phi_hi = nullptr;
  const __nv_bfloat16* phi_lo = nullptr;
  const int32_t* edges = nullptr;
  const DstItem* items = nullptr;
  int32_t n_items = 0;
  int32_t sp = 0;
};
// Samples padded to a power of two >= 8 (0 if S > 256: no tensor-core path).
int32_t dst_gemm_sample_pad(int64_t S);
int32_t dst_gemm_tile_rows();
int32_t dst_gemm_tile_k();
int32_t dst_gemm_tile_cols();
void launch_phi_planes(const DstGroup* groups, int32_t n_groups, __nv_bfloat16* hi,
                       __nv_bfloat16* lo, cudaStream_t st);
// kInv = false: dst = bhat [n_interior][S] from src = b [n][S] (noise rows);
// kInv = true: dst = out [S][n] (interior DOFs) from src = c [n_interior][S].
// A timed-out wait adds to status->device_timeout.
template <bool kInv, typename OutT>
int launch_dst_gemm(const DevGraph& g, const DstPlanDev& p, int64_t S, const float* src,
                    OutT* dst, PcgStatus* status, int n_sm, cudaStream_t st);

// ---- recover.cu
// Edge bins of the register-resident recovery: bin i takes edges with
// m <= 32 * NW[i] * B[i] interior nodes. Returns the number of bins.
constexpr int kMaxBins = 8;
int recover_bins(bool fp64, int32_t* B, int32_t* NW);
// bin_edges: edge ids grouped by bin (bin_count[i] each, bins in order);
// prm[l][e] sweep constants, xw[l][v][s] = w_l u_v^(l) in precision T.
// Returns the number of kernels launched.
// sg: samples per lane (FP32 sweeps: 1, 2 or 4; FP64 sweeps use 2).
template <typename T, typename OutT>
int launch_recover_bins(const DevGraph& g, int32_t L, int64_t S, const T* b,
                        const SweepParams<T>* prm, const T* xw, OutT* out,
                        const int32_t* bin_edges, const int32_t* bin_count, int sg,
                        cudaStream_t st);

}  // namespace grf
