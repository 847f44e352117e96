// C ABI of the sampler (include/grf.h): graph building, quadrature nodes,
// workspace management and the launch sequence of one sample call.
//
// Launch sequence of grf_sample (Sec. 3, Phases 2-5):
//   noise (Phase 2) -> per node l: 2x2 edge Schur blocks and vertex diagonal
//   -> condensed right-hand side g (Phase 3) -> Jacobi-PCG per (l, s)
//   (Phase 4) -> vertex quadrature sum and fused interior recovery +
//   quadrature sum (Phase 5). All nodes and samples are batched in each launch.
#include <cmath>
#include <cstdarg>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/grf.h"
#include "grf_internal.h"

using namespace grf;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      return fail(_e == cudaErrorMemoryAllocation ? GRF_ENOMEM : GRF_ECUDA, "%s: %s (%s:%d)", \
                  #expr, cudaGetErrorString(_e), __FILE__, __LINE__);                    \
  } while (0)

#define GRF_TRY(expr)       \
  do {                      \
    int _r = (expr);        \
    if (_r != GRF_OK) return _r; \
  } while (0)

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Bump allocator over one cached device block.
struct Carve {
  char* base;
  size_t off = 0;
  bool dry;
  explicit Carve(void* b) : base((char*)b), dry(b == nullptr) {}
  template <typename T>
  T* take(size_t count) {
    size_t o = off;
    off += align_up(count * sizeof(T));
    return dry ? nullptr : reinterpret_cast<T*>(base + o);
  }
};

// Learned B B^T preconditioner state kept on a graph handle: FP32 master
// weights, their BF16 copies (layers and transposed layers), Adam moments, a
// gradient accumulator, a node-index ramp and per-step loss slots.
constexpr int kRamp = 1 << 16;
struct LearnedModel {
  void* blk = nullptr;
  float *P = nullptr, *G = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *wb = nullptr, *wt = nullptr;
  int32_t* ramp = nullptr;  // 0, 1, ..., kRamp - 1
  int step = 0;             // Adam steps taken since the weights were set
  bool ready = false;
};

}  // namespace

// One timed phase of a call: CUDA events recorded on the call's stream before
// and after it (phase index as in grf_stats.phase_ms).
struct PhaseSpan {
  int phase;
  cudaEvent_t a, b;
};

struct grf_graph {
  int64_t nv_in = 0;
  int32_t nv = 0;
  int32_t ne = 0;
  int64_t ni = 0;
  int64_t n = 0;
  std::vector<int64_t> vertex_map;
  std::vector<int32_t> eu, ev, nel, vptr, adj_edge, adj_nbr, adj_rev;
  // the vertices in reverse Cuthill-McKee order (slot -> vertex) and the
  // incidence lists in that order: neighbour slot and original incidence index
  std::vector<int32_t> rperm, rvptr, rnbr, rinc;
  VertexOrder d_order{};
  std::vector<double> he;
  std::vector<int64_t> ioff;
  std::vector<double> ml_vertex;  // lumped mass at kept vertices
  // Thomas recovery edge bins ([0] FP32 sweeps, [1] FP64, [2] FP32 sweeps of the
  // edges the spectral path leaves to Thomas): edge ids grouped by bin, the
  // count per bin, and last the edges beyond every bin
  std::vector<int32_t> bin_edges[3];
  int32_t bin_count[3][kMaxBins + 1] = {};
  int32_t n_bins[3] = {0, 0, 0};
  const int32_t* d_bin_edges[3] = {nullptr, nullptr, nullptr};
  // spectral bins (edges with 1 <= m <= the largest spectral bin)
  std::vector<int32_t> spec_edges;
  int32_t spec_count[kMaxBins] = {};
  int32_t n_spec_bins = 0;
  const int32_t* d_spec_edges = nullptr;

  int64_t long_edges(bool fp64) const { return bin_count[fp64 ? 1 : 0][n_bins[fp64 ? 1 : 0]]; }
  int64_t thomas_rest() const {  // edges of bins [2]
    int64_t n = 0;
    for (int i = 0; i <= n_bins[2]; ++i) n += bin_count[2][i];
    return n;
  }

  int device = -1;
  int n_sm = 0;  // multiprocessors of that device
  const float* d_sqrt_ml_f = nullptr;  // FP32 copy of DevGraph::sqrt_ml (FP32 noise)
  // per vertex its first four neighbours (int4, padded with itself), then per
  // vertex the start of its incidence list and its degree (int2): the batched
  // PCG's gathers
  const int4* d_ell = nullptr;
  void* dev_block = nullptr;
  // Cholesky factor of the consistent mass's vertex Schur complement (CSR,
  // FP32 on the device; built on first use of the consistent mass)
  struct ConsPlan {
    void* blk = nullptr;
    const int64_t* rp = nullptr;
    const int32_t* rc = nullptr;
    const float* rv = nullptr;
    const float* ones = nullptr;  // unit mass factors: the noise kernel's raw normals
  } cons;
  // sine-transform plan of the tensor-core spectral path (built on first use,
  // for one sample padding at a time)
  struct DstPlan {
    void* blk = nullptr;
    DstPlanDev dev{};
  } dst;
  DevGraph d{};
  void* ws = nullptr;
  size_t ws_bytes = 0;

  // Captured launch sequence of one grf_sample configuration (options.use_graph).
  // Device pointers (workspace, output, node arrays) are baked into the graph,
  // so any change of them or of the configuration re-captures.
  struct GraphCache {
    bool valid = false;
    int precision = 0, precond = 0, out_dtype = 0, pcg_layout = 0, recover_sg = 0, max_iter = 0;
    bool spectral = false, spec_tc = false, spec_umma = false, consistent = false, timing = false;
    uint32_t phase_mask = 0;
    int sweep = 0;
    double rtol = 0, kappa = 0, beta = 0, k = 0;
    int64_t S = 0;
    void* out = nullptr;
    void* ws = nullptr;
    cudaGraphExec_t exec = nullptr;
    double* nodes_dev = nullptr;   // per stage alpha|gamma|weight, then the seed word
    uint64_t* d_seed = nullptr;
    uint64_t* h_seed = nullptr;    // pinned
    PcgStatus* h_status = nullptr; // pinned, one per stage
    int h_status_cap = 0;
    std::vector<int32_t> stage_L;
    int launches = 0;
    // with phase timing: the phase events, nodes of the graph that every
    // replay records again
    std::vector<PhaseSpan> spans;
  } gc;
  cudaStream_t cap_stream = nullptr;
  LearnedModel lm;
  // device output of grf_sample_host, kept between calls so that a captured
  // CUDA graph (which bakes the output pointer in) stays valid
  void* host_out = nullptr;
  size_t host_out_bytes = 0;
  // grf_sample_host_stream: the second device buffer, the copy stream and its
  // two events (the staged field, the finished host copy)
  void* host_stage = nullptr;
  size_t host_stage_bytes = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_staged = nullptr, ev_d2h = nullptr;
  // the Schur blocks' side stream and its fork and join events
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  void drop_graph() {
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    if (gc.nodes_dev) cudaFree(gc.nodes_dev);
    for (auto& sp : gc.spans) {
      cudaEventDestroy(sp.a);
      cudaEventDestroy(sp.b);
    }
    gc.spans.clear();
    gc.exec = nullptr;
    gc.nodes_dev = nullptr;
    gc.d_seed = nullptr;
    gc.valid = false;
  }

  ~grf_graph() {
    if (device >= 0) {
      int cur = 0;
      cudaGetDevice(&cur);
      cudaSetDevice(device);
      drop_graph();
      if (gc.h_seed) cudaFreeHost(gc.h_seed);
      if (gc.h_status) cudaFreeHost(gc.h_status);
      if (cap_stream) cudaStreamDestroy(cap_stream);
      if (dev_block) cudaFree(dev_block);
      if (ws) cudaFree(ws);
      if (lm.blk) cudaFree(lm.blk);
      if (host_out) cudaFree(host_out);
      if (host_stage) cudaFree(host_stage);
      if (ev_staged) cudaEventDestroy(ev_staged);
      if (ev_d2h) cudaEventDestroy(ev_d2h);
      if (copy_stream) cudaStreamDestroy(copy_stream);
      if (ev_fork) cudaEventDestroy(ev_fork);
      if (ev_join) cudaEventDestroy(ev_join);
      if (side_stream) cudaStreamDestroy(side_stream);
      if (dst.blk) cudaFree(dst.blk);
      if (cons.blk) cudaFree(cons.blk);
      cudaSetDevice(cur);
    }
  }
};

namespace {

__global__ void sqrt_ml_kernel(DevGraph g, const double* mlv, double* out, float* out_f) {
  const int64_t total = g.n;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total;
       j += (int64_t)gridDim.x * blockDim.x) {
    if (j < g.nv) {
      out[j] = sqrt(mlv[j]);
      out_f[j] = (float)out[j];
    } else {
      // interior DOF: find its edge by bisection over the interior offsets
      const int64_t i = j - g.nv;
      int32_t lo = 0, hi = g.ne - 1;
      while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (g.ioff[mid] <= i) lo = mid; else hi = mid - 1;
      }
      out[j] = sqrt(g.he[lo]);
      out_f[j] = (float)out[j];
    }
  }
}

int ensure_device(grf_graph* g) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (g->device == dev && g->dev_block) return GRF_OK;
  if (g->device >= 0 && g->device != dev)
    return fail(GRF_EINVAL, "graph was first used on device %d, now on device %d", g->device, dev);
  const size_t E = (size_t)g->ne, V = (size_t)g->nv;
  Carve c(nullptr);
  c.take<int32_t>(E); c.take<int32_t>(E); c.take<int32_t>(E); c.take<double>(E);
  c.take<int64_t>(E + 1); c.take<int32_t>(V + 1); c.take<int32_t>(2 * E); c.take<int32_t>(2 * E);
  c.take<double>((size_t)g->n); c.take<double>(V);
  c.take<int32_t>(E + 1); c.take<int32_t>(E + 1); c.take<int32_t>(E + 1); c.take<int32_t>(E + 1);
  c.take<int32_t>(2 * E);
  c.take<int32_t>(V); c.take<int32_t>(V + 1); c.take<int32_t>(2 * E); c.take<int32_t>(2 * E);
  c.take<float>((size_t)g->n);
  c.take<int4>(2 * V);
  c.take<int4>(V); c.take<int32_t>(V);
  void* blk = nullptr;
  CUDA_TRY(cudaMalloc(&blk, c.off));
  g->device = dev;
  g->dev_block = blk;
  CUDA_TRY(cudaDeviceGetAttribute(&g->n_sm, cudaDevAttrMultiProcessorCount, dev));
  Carve k(blk);
  int32_t* eu = k.take<int32_t>(E);
  int32_t* ev = k.take<int32_t>(E);
  int32_t* nel = k.take<int32_t>(E);
  double* he = k.take<double>(E);
  int64_t* ioff = k.take<int64_t>(E + 1);
  int32_t* vptr = k.take<int32_t>(V + 1);
  int32_t* ae = k.take<int32_t>(2 * E);
  int32_t* an = k.take<int32_t>(2 * E);
  double* sml = k.take<double>((size_t)g->n);
  double* mlv = k.take<double>(V);
  for (int p = 0; p < 3; ++p) {
    int32_t* be = k.take<int32_t>(E + 1);
    if (!g->bin_edges[p].empty())
      CUDA_TRY(cudaMemcpy(be, g->bin_edges[p].data(), g->bin_edges[p].size() * 4,
                          cudaMemcpyHostToDevice));
    g->d_bin_edges[p] = be;
  }
  {
    int32_t* se = k.take<int32_t>(E + 1);
    if (!g->spec_edges.empty())
      CUDA_TRY(cudaMemcpy(se, g->spec_edges.data(), g->spec_edges.size() * 4,
                          cudaMemcpyHostToDevice));
    g->d_spec_edges = se;
  }
  CUDA_TRY(cudaMemcpy(eu, g->eu.data(), E * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(ev, g->ev.data(), E * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(nel, g->nel.data(), E * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(he, g->he.data(), E * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(ioff, g->ioff.data(), (E + 1) * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(vptr, g->vptr.data(), (V + 1) * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(ae, g->adj_edge.data(), 2 * E * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(an, g->adj_nbr.data(), 2 * E * 4, cudaMemcpyHostToDevice));
  int32_t* arev = k.take<int32_t>(2 * E);
  CUDA_TRY(cudaMemcpy(arev, g->adj_rev.data(), 2 * E * 4, cudaMemcpyHostToDevice));
  int32_t* rperm = k.take<int32_t>(V);
  int32_t* rvptr = k.take<int32_t>(V + 1);
  int32_t* rnbr = k.take<int32_t>(2 * E);
  int32_t* rinc = k.take<int32_t>(2 * E);
  CUDA_TRY(cudaMemcpy(rperm, g->rperm.data(), V * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(rvptr, g->rvptr.data(), (V + 1) * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(rnbr, g->rnbr.data(), 2 * E * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(rinc, g->rinc.data(), 2 * E * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(mlv, g->ml_vertex.data(), V * 8, cudaMemcpyHostToDevice));
  DevGraph& d = g->d;
  d.nv = g->nv; d.ne = g->ne; d.ni = g->ni; d.n = g->n;
  d.max_m = 0;
  for (int32_t e = 0; e < g->ne; ++e) d.max_m = std::max(d.max_m, g->nel[e] - 1);
  d.eu = eu; d.ev = ev; d.nel = nel; d.he = he; d.ioff = ioff;
  d.vptr = vptr; d.adj_edge = ae; d.adj_nbr = an; d.adj_rev = arev; d.sqrt_ml = sml;
  g->d_order = VertexOrder{rperm, rvptr, rnbr, rinc};
  int64_t blocks = (g->n + 255) / 256;
  if (blocks > sm_count() * 32) blocks = sm_count() * 32;
  float* smlf = k.take<float>((size_t)g->n);
  g->d_sqrt_ml_f = smlf;
  {
    // V int4 (neighbours) then V int2 (incidence-list start, degree)
    int4* ell = k.take<int4>(2 * V);
    std::vector<int4> h(2 * V);
    int2* info = reinterpret_cast<int2*>(h.data() + V);
    for (size_t v = 0; v < V; ++v) {
      const int32_t k0 = g->vptr[v], deg = g->vptr[v + 1] - k0;
      int32_t w[4];
      for (int i = 0; i < 4; ++i) w[i] = i < deg ? g->adj_nbr[k0 + i] : (int32_t)v;
      h[v] = make_int4(w[0], w[1], w[2], w[3]);
      info[v] = make_int2(k0, deg);
    }
    CUDA_TRY(cudaMemcpy(ell, h.data(), 2 * V * sizeof(int4), cudaMemcpyHostToDevice));
    g->d_ell = ell;
    // the end-value gather's records: incidences on sine-basis edges
    int4* sinc = k.take<int4>(V);
    int32_t* scnt = k.take<int32_t>(V);
    std::vector<int4> hs(V);
    std::vector<int32_t> hc(V);
    for (size_t v = 0; v < V; ++v) {
      int32_t w[4] = {-1, -1, -1, -1}, c = 0;
      for (int32_t kk = g->vptr[v]; kk < g->vptr[v + 1]; ++kk) {
        const int32_t e = g->adj_edge[kk], m = g->nel[e] - 1;
        if (m < 1 || m > kSpecMaxM) continue;
        if (c < 4) w[c] = 2 * e + (g->eu[e] == (int64_t)v ? 0 : 1);
        ++c;
      }
      hs[v] = make_int4(w[0], w[1], w[2], w[3]);
      hc[v] = c;
    }
    CUDA_TRY(cudaMemcpy(sinc, hs.data(), V * sizeof(int4), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(scnt, hc.data(), V * sizeof(int32_t), cudaMemcpyHostToDevice));
    d.spec_inc = sinc;
    d.spec_cnt = scnt;
  }
  sqrt_ml_kernel<<<(int)blocks, 256>>>(d, mlv, sml, smlf);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaDeviceSynchronize());
  return GRF_OK;
}

int ensure_ws(grf_graph* g, size_t bytes) {
  if (g->ws && g->ws_bytes >= bytes) return GRF_OK;
  if (g->ws) {
    CUDA_TRY(cudaDeviceSynchronize());
    g->drop_graph();  // the captured graph refers to the old workspace
    CUDA_TRY(cudaFree(g->ws));
    g->ws = nullptr;
    g->ws_bytes = 0;
  }
  CUDA_TRY(cudaMalloc(&g->ws, bytes));
  g->ws_bytes = bytes;
  return GRF_OK;
}

// The tensor-core sine transforms (interior GRF_INTERIOR_SPECTRAL_UMMA): the
// spectral edges grouped by interior-node count m, Phi_m's BF16 hi/lo planes
// and the work items for sample padding sp. Built before any capture, for one
// sp at a time (S > 256 has no plan: the call takes the FP32 spectral kernels).
int ensure_dst_plan(grf_graph* g, int64_t S) {
  const int32_t sp = dst_gemm_sample_pad(S);
  if (sp == 0) return GRF_OK;
  if (g->dst.blk && g->dst.dev.sp == sp) return GRF_OK;
  if (g->dst.blk) {
    CUDA_TRY(cudaDeviceSynchronize());
    g->drop_graph();  // a captured graph refers to the old plan
    CUDA_TRY(cudaFree(g->dst.blk));
    g->dst = grf_graph::DstPlan{};
  }
  const int32_t BM = dst_gemm_tile_rows(), BK = dst_gemm_tile_k(), BN = dst_gemm_tile_cols();
  const int32_t ept = BN / sp;
  std::map<int32_t, std::vector<int32_t>> by_m;
  for (int32_t e : g->spec_edges) by_m[g->nel[e] - 1].push_back(e);
  std::vector<DstGroup> groups;
  std::vector<DstItem> items;
  std::vector<int32_t> edges;
  int64_t phi_total = 0;
  for (auto& kv : by_m) {
    const int32_t m = kv.first;
    const std::vector<int32_t>& list = kv.second;
    DstGroup G{phi_total, m, (m + BM - 1) / BM * BM, (m + BK - 1) / BK * BK, 0};
    groups.push_back(G);
    const int32_t e0 = (int32_t)edges.size();
    edges.insert(edges.end(), list.begin(), list.end());
    for (int32_t t = 0; t < (int32_t)list.size(); t += ept)
      for (int32_t mt = 0; mt < G.mp / BM; ++mt)
        items.push_back(DstItem{G.phi_off, m, G.kp, e0 + t,
                                std::min<int32_t>(ept, (int32_t)list.size() - t), mt, 0});
    phi_total += (int64_t)G.mp * G.kp;
  }
  if (items.empty()) return GRF_OK;
  Carve dry(nullptr);
  dry.take<__nv_bfloat16>(phi_total);
  dry.take<__nv_bfloat16>(phi_total);
  dry.take<int32_t>(edges.size());
  dry.take<DstGroup>(groups.size());
  dry.take<DstItem>(items.size());
  void* blk = nullptr;
  CUDA_TRY(cudaMalloc(&blk, dry.off));
  Carve c(blk);
  __nv_bfloat16* hi = c.take<__nv_bfloat16>(phi_total);
  __nv_bfloat16* lo = c.take<__nv_bfloat16>(phi_total);
  int32_t* de = c.take<int32_t>(edges.size());
  DstGroup* dg = c.take<DstGroup>(groups.size());
  DstItem* di = c.take<DstItem>(items.size());
  CUDA_TRY(cudaMemcpy(de, edges.data(), edges.size() * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(dg, groups.data(), groups.size() * sizeof(DstGroup), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(di, items.data(), items.size() * sizeof(DstItem), cudaMemcpyHostToDevice));
  launch_phi_planes(dg, (int32_t)groups.size(), hi, lo, 0);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaDeviceSynchronize());
  g->dst.blk = blk;
  g->dst.dev = DstPlanDev{hi, lo, de, di, (int32_t)items.size(), sp};
  return GRF_OK;
}

struct HostNodes {
  std::vector<double> alpha, gamma, weight;
  int32_t L() const { return (int32_t)alpha.size(); }
};

// w_l A_l^{-1} = (w_l / s_l) (A_l / s_l)^{-1} for any s_l > 0: every node is
// rescaled by s_l = max(alpha_l, gamma_l), exactly in FP64 on the host, so that
// the shifted operator's coefficients and the weights that reach the FP32
// kernels stay O(1) whatever the shift (e^{2y} passes the FP32 range for the
// outer sinc nodes of small steps: 3.4e38 at y = 44.4).
void normalize_nodes(HostNodes& h) {
  for (size_t l = 0; l < h.alpha.size(); ++l) {
    const double s = std::max(h.alpha[l], h.gamma[l]);
    if (s > 0 && std::isfinite(s)) {
      h.alpha[l] /= s;
      h.gamma[l] /= s;
      h.weight[l] /= s;
    }
  }
}

// Sinc quadrature nodes of Eq. 4 with the limits of Sec. 4.1, 0 < f < 1:
// y_l = l k, l = -K^- .. K^+; A_l = M_L + t_l K with t_l = e^{2 y_l};
// weight w_l = (2 k sin(pi f) / pi) e^{2 f y_l}.
HostNodes quadrature_nodes(double f, double k) {
  const double pi = 3.14159265358979323846;
  const long km = (long)std::ceil(pi * pi / (4.0 * k * k * f));
  const long kp = (long)std::ceil(pi * pi / (4.0 * k * k * (1.0 - f)));
  HostNodes h;
  const double c = 2.0 * k * std::sin(pi * f) / pi;
  for (long l = -km; l <= kp; ++l) {
    const double y = (double)l * k;
    h.alpha.push_back(1.0);
    h.gamma.push_back(std::exp(2.0 * y));
    h.weight.push_back(c * std::exp(2.0 * f * y));
  }
  normalize_nodes(h);
  return h;
}

HostNodes stiffness_node() {
  HostNodes h;
  h.alpha.push_back(0.0);
  h.gamma.push_back(1.0);
  h.weight.push_back(1.0);
  return h;
}

struct Opts {
  int precision, precond, out_dtype, max_iter;
  double rtol;
  bool timing;
  uint32_t phase_mask;  // phases timed (bit p = grf_stats.phase_ms[p]) when timing
  int pcg_layout;  // 1 per system, 2 staged
  int recover_sg;  // 1, 2 or 4
  bool use_graph;
  bool spectral;   // edge interiors in the sine basis (mixed precision)
  bool spec_tc;    // ... with the transforms and contractions on the tensor cores
  bool spec_umma;  // ... with the sine transforms as tcgen05 products per edge length
  bool consistent; // the consistent-mass comparison system (noise and operator)
  int sweep;       // GRF_SWEEP_* of the FP32 tridiagonal edges
};

int read_opts(const grf_options* o, Opts* r) {
  r->use_graph = o && o->use_graph != 0;
  r->timing = o && o->timing != 0;
  r->phase_mask = 0xFFu;
  if (r->timing && (o->timing & GRF_TIMING_ONLY)) {
    const uint32_t t = (uint32_t)o->timing;
    if ((t & ~(uint32_t)GRF_TIMING_ONLY & ~0xFFu) != 0 || (t & 0xFFu) == 0)
      return fail(GRF_EINVAL, "timing: GRF_TIMING_ONLY needs a phase mask in bits 0-7 (got 0x%x)",
                  t);
    r->phase_mask = t & 0xFFu;
  }
  const int sg = o ? o->recover_sg : 0;
  if (sg != 0 && sg != 1 && sg != 2 && sg != 4)
    return fail(GRF_EINVAL, "recover_sg must be 0, 1, 2 or 4 (got %d)", sg);
  r->recover_sg = sg == 0 ? 4 : sg;
  const int lay = o ? o->pcg_layout : GRF_PCG_AUTO;
  if (lay < GRF_PCG_AUTO || lay > GRF_PCG_BATCHED)
    return fail(GRF_EINVAL, "unknown pcg_layout %d", lay);
  // AUTO: the sample-group layout where it applies (launch_pcg falls back to
  // one CTA per system otherwise)
  r->pcg_layout = lay == GRF_PCG_AUTO ? GRF_PCG_STAGED : lay;
  r->precision = o ? o->precision : GRF_FP64;
  r->precond = o ? o->precond : GRF_PRECOND_JACOBI;
  r->out_dtype = o ? o->out_dtype : GRF_OUT_F64;
  r->max_iter = (o && o->max_iter > 0) ? o->max_iter : 1000;
  r->rtol = (o && o->rtol > 0) ? o->rtol : (r->precision == GRF_FP64 ? 1e-12 : 1e-8);
  if (r->precision != GRF_FP64 && r->precision != GRF_MIXED)
    return fail(GRF_EINVAL, "unknown precision %d", r->precision);
  if (r->precond != GRF_PRECOND_JACOBI && r->precond != GRF_PRECOND_LEARNED &&
      r->precond != GRF_PRECOND_NEUMANN)
    return fail(GRF_ENOTSUP, "preconditioner %d not available", r->precond);
  if (r->precond == GRF_PRECOND_LEARNED && r->precision != GRF_MIXED)
    return fail(GRF_ENOTSUP, "the learned preconditioner needs precision GRF_MIXED");
  if (r->out_dtype != GRF_OUT_F64 && r->out_dtype != GRF_OUT_F32)
    return fail(GRF_EINVAL, "unknown out_dtype %d", r->out_dtype);
  const int in = o ? o->interior : GRF_INTERIOR_AUTO;
  if (in < GRF_INTERIOR_AUTO || in > GRF_INTERIOR_SPECTRAL_UMMA)
    return fail(GRF_EINVAL, "unknown interior solver %d", in);
  if ((in == GRF_INTERIOR_SPECTRAL || in == GRF_INTERIOR_SPECTRAL_TC ||
       in == GRF_INTERIOR_SPECTRAL_UMMA) && r->precision != GRF_MIXED)
    return fail(GRF_ENOTSUP, "the spectral interior solver needs precision GRF_MIXED");
  r->spectral = r->precision == GRF_MIXED && in != GRF_INTERIOR_THOMAS;
  r->spec_tc = r->spectral && in == GRF_INTERIOR_SPECTRAL_TC;
  r->spec_umma = r->spectral && in == GRF_INTERIOR_SPECTRAL_UMMA;
  const int mass = o ? o->mass : GRF_MASS_LUMPED;
  if (mass != GRF_MASS_LUMPED && mass != GRF_MASS_CONSISTENT)
    return fail(GRF_EINVAL, "unknown mass %d", mass);
  r->consistent = mass == GRF_MASS_CONSISTENT;
  if (r->consistent) {
    if (r->precision != GRF_MIXED || r->precond != GRF_PRECOND_JACOBI ||
        (in != GRF_INTERIOR_AUTO && in != GRF_INTERIOR_SPECTRAL_UMMA))
      return fail(GRF_ENOTSUP,
                  "the consistent mass runs with precision GRF_MIXED, GRF_PRECOND_JACOBI and "
                  "the interior solver AUTO or SPECTRAL_UMMA");
    r->spec_umma = r->spectral;
  }
  r->sweep = o ? o->sweep : GRF_SWEEP_AUTO;
  if (r->sweep < GRF_SWEEP_AUTO || r->sweep > GRF_SWEEP_NODES)
    return fail(GRF_EINVAL, "unknown sweep layout %d", r->sweep);
  return GRF_OK;
}

// Consistent-mass noise, set-up (once per graph): the vertex Schur complement
// of the consistent mass, S_M = M_GG - M_GI M_II^-1 M_IG, from per-edge 2x2
// blocks (on an edge M_II = tridiag(h/6, 2h/3, h/6) with the vertex couplings
// h/6 and the edge's share h/3 of M_vv; with r = h/6 and cosh(theta) = 2 the
// block is r sinh(theta) [[coth(n theta), (-1)^(n+1) csch(n theta)], ...]),
// then its Cholesky factor in kept-vertex order by an envelope (skyline)
// factorisation: row i holds columns first(i) .. i, first(i) its lowest
// neighbour, and the fill stays inside the envelope. Refused above 2^27
// envelope entries (the consistent mass of a graph without a narrow vertex
// numbering: what makes the comparison system expensive).
int ensure_cons_plan(grf_graph* g) {
  if (g->cons.blk) return GRF_OK;
  GRF_TRY(ensure_device(g));
  const int32_t V = g->nv;
  std::vector<double> diag(V, 0.0);
  std::vector<int32_t> first(V);
  for (int32_t v = 0; v < V; ++v) first[v] = v;
  const double th = std::acosh(2.0), sh = std::sinh(th);
  std::map<std::pair<int32_t, int32_t>, double> off;
  for (int32_t e = 0; e < g->ne; ++e) {
    const double r = g->he[e] / 6.0;
    const int32_t n = g->nel[e];
    const double q = std::exp(-(double)n * th);  // e^{-n theta}
    const double coth = (1.0 + q * q) / (1.0 - q * q), csch = 2.0 * q / (1.0 - q * q);
    const int32_t u = g->eu[e], v = g->ev[e];
    diag[u] += r * sh * coth;
    diag[v] += r * sh * coth;
    const double b = ((n & 1) ? 1.0 : -1.0) * r * sh * csch;
    const int32_t lo = std::min(u, v), hi = std::max(u, v);
    off[{hi, lo}] += b;
    first[hi] = std::min(first[hi], lo);
  }
  std::vector<int64_t> rp(V + 1, 0);
  for (int32_t i = 0; i < V; ++i) rp[i + 1] = rp[i] + (i - first[i] + 1);
  const int64_t nnz = rp[V];
  if (nnz > ((int64_t)1 << 27))
    return fail(GRF_ENOTSUP,
                "the consistent-mass factor of this graph needs %lld envelope entries "
                "(limit 2^27); number the vertices with a narrower band",
                (long long)nnz);
  std::vector<double> L((size_t)nnz, 0.0);
  auto at = [&](int32_t i, int32_t j) -> double& { return L[(size_t)(rp[i] + (j - first[i]))]; };
  for (int32_t i = 0; i < V; ++i) at(i, i) = diag[i];
  for (auto& kv : off) at(kv.first.first, kv.first.second) = kv.second;
  for (int32_t i = 0; i < V; ++i) {
    for (int32_t j = first[i]; j < i; ++j) {
      double acc = at(i, j);
      const int32_t k0 = std::max(first[i], first[j]);
      const double* li = &L[(size_t)(rp[i] + (k0 - first[i]))];
      const double* lj = &L[(size_t)(rp[j] + (k0 - first[j]))];
      for (int32_t k = 0; k < j - k0; ++k) acc -= li[k] * lj[k];
      at(i, j) = acc / at(j, j);
    }
    double acc = at(i, i);
    for (int32_t k = first[i]; k < i; ++k) acc -= at(i, k) * at(i, k);
    if (!(acc > 0.0)) return fail(GRF_ENUMERIC, "consistent-mass factor: pivot %d is %g", i, acc);
    at(i, i) = std::sqrt(acc);
  }
  std::vector<int32_t> rc((size_t)nnz);
  std::vector<float> rv((size_t)nnz);
  for (int32_t i = 0; i < V; ++i)
    for (int32_t j = first[i]; j <= i; ++j) {
      rc[(size_t)(rp[i] + (j - first[i]))] = j;
      rv[(size_t)(rp[i] + (j - first[i]))] = (float)at(i, j);
    }
  Carve dry(nullptr);
  dry.take<int64_t>(V + 1);
  dry.take<int32_t>((size_t)nnz);
  dry.take<float>((size_t)nnz);
  dry.take<float>((size_t)g->n);
  void* blk = nullptr;
  CUDA_TRY(cudaMalloc(&blk, dry.off));
  Carve c(blk);
  int64_t* drp = c.take<int64_t>(V + 1);
  int32_t* drc = c.take<int32_t>((size_t)nnz);
  float* drv = c.take<float>((size_t)nnz);
  float* ones = c.take<float>((size_t)g->n);
  CUDA_TRY(cudaMemcpy(drp, rp.data(), sizeof(int64_t) * (V + 1), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(drc, rc.data(), sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(drv, rv.data(), sizeof(float) * (size_t)nnz, cudaMemcpyHostToDevice));
  std::vector<float> one((size_t)g->n, 1.0f);
  CUDA_TRY(cudaMemcpy(ones, one.data(), sizeof(float) * (size_t)g->n, cudaMemcpyHostToDevice));
  g->cons.blk = blk;
  g->cons.rp = drp;
  g->cons.rc = drc;
  g->cons.rv = drv;
  g->cons.ones = ones;
  return GRF_OK;
}

// The consistent mass needs every edge on the sine-basis path and a
// fractional beta (the integer part would need the consistent mass between
// the stiffness solves).
int check_consistent(const grf_graph* g, const Opts& o, double beta, int64_t S) {
  if (!o.consistent) return GRF_OK;
  if (g->thomas_rest() > 0)
    return fail(GRF_ENOTSUP, "the consistent mass needs every edge within 1024 interior nodes");
  if (beta >= 1.0) return fail(GRF_ENOTSUP, "the consistent mass runs with 0 < beta < 1");
  if (dst_gemm_sample_pad(S) == 0)
    return fail(GRF_ENOTSUP, "the consistent mass runs with at most 256 samples per call");
  return GRF_OK;
}

// The FP32 edge-interior kernels work with delta_l = (alpha_l / gamma_l +
// kappa^2) h_e^2 and c_l = gamma_l / h_e (nodes already rescaled to
// max(alpha, gamma) = 1). Nodes whose delta passes 1e36 or whose c falls below
// 1e-36 on some edge (shifts t_l below about 1e-36 h) leave the FP32 range
// (normal numbers down to 1.2e-38) and are refused in mixed precision; FP64
// takes them. The sinc nodes of k = 0.25, beta = 0.25 on h = 2^-9 reach
// delta 8e28 and c 3e-32.
int check_fp32_range(const grf_graph* g, const Opts& o, double kappa,
                     const std::vector<HostNodes>& stages) {
  if (o.precision == GRF_FP64 || g->ne == 0) return GRF_OK;
  double hmax = 0.0;
  for (int32_t e = 0; e < g->ne; ++e) hmax = std::max(hmax, g->he[e]);
  for (auto& s : stages)
    for (int32_t l = 0; l < s.L(); ++l) {
      if (!(s.gamma[l] > 0)) continue;
      const double delta = (s.alpha[l] / s.gamma[l] + kappa * kappa) * hmax * hmax;
      const double c = s.gamma[l] / hmax;
      if (!(delta < 1e36) || !(c > 1e-36))
        return fail(GRF_ENOTSUP,
                    "quadrature node %d (alpha %g, gamma %g) is outside the FP32 range of the "
                    "mixed path on this mesh (delta %g, c %g); use FP64",
                    (int)l, s.alpha[l], s.gamma[l], delta, c);
    }
  return GRF_OK;
}

// The tensor-core transforms run for this call (the plan exists for its S).
bool umma_ready(const grf_graph* g, const Opts& o, int64_t S, int32_t L) {
  return o.spec_umma && g->dst.blk && g->dst.dev.sp == dst_gemm_sample_pad(S) &&
         g->dst.dev.n_items > 0 && spec_umma_fits(L);
}

// FP32 tridiagonal edges of path p (0: every edge, 2: the edges the spectral
// path leaves over) are grouped by recovery bin in increasing length. The edges
// from bin node_bin0 on (and those beyond every bin) are swept by the
// node-parallel kernels. AUTO (measured on GB300 with 148 nodes and 64
// samples): from about 100 interior nodes on they condense 1.5-3x and recover
// 1.7-3.6x faster than the segment kernels.
int node_bin0(const grf_graph* g, int p, const Opts& o, int32_t L) {
  const int nb = g->n_bins[p];
  if (o.sweep == GRF_SWEEP_SEGMENTS || !node_sweep_fits(L)) return nb + 1;
  if (o.sweep == GRF_SWEEP_NODES) return 0;
  int32_t B[kMaxBins], NW[kMaxBins];
  recover_bins(false, B, NW);
  int32_t lo = 0;  // bin i holds lo < m <= 32 NW B
  for (int i = 0; i < nb; ++i) {
    if (lo >= 64) return i;
    lo = 32 * NW[i] * B[i];
  }
  return nb;
}
int32_t bins_before(const grf_graph* g, int p, int i0) {
  int32_t n = 0;
  for (int i = 0; i < i0 && i <= g->n_bins[p]; ++i) n += g->bin_count[p][i];
  return n;
}
int32_t bins_total(const grf_graph* g, int p) { return bins_before(g, p, g->n_bins[p] + 1); }

// Device workspace of one domain-decomposed apply with L nodes and S right-hand sides.
struct ApplyWs {
  double *alpha, *gamma, *weight, *saa, *sab, *diag, *offv, *gvec, *x, *acc;
  void *r, *p, *q, *d, *y;  // PCG vectors in the sweep precision T [L][S][V]
  void *pre_c, *pre_n;      // preconditioner coefficients per node: [L][V], [L][2E]
                            // (learned: float es, N; Neumann-Neumann: T)
  LpActs lpa;               // network activations of lp_chunk nodes (es, n set per chunk)
  int32_t lp_chunk;
  void* dscale;         // T [L][V]
  void* offv_t;         // float [L][2E] (mixed precision only)
  float2 *dpair, *opair;  // FP64 blocks as FP32 pairs [L][V], [L][2E] (mixed only)
  float *xh, *xl, *gh, *gl;  // batched PCG refinement vectors, shaped as r (mixed only)
  void *yscr, *rpscr;
  void* prm;  // SweepParams<T> [L][E]
  void* xw;   // T [L][V][S] (sample-minor)
  float* bhat;  // sine transform of the interior noise [n_interior][S] (spectral path)
  float* ends;  // end values per edge [E][2][S][L] (tensor-core sine-basis path)
  float *nshift, *nwgam;  // FP32 node constants [L] (spectral path)
  int32_t* iters;
  PcgStatus* status;
};

// Nodes per network pass when the learned preconditioner runs inside a sample
// call: about 2^20 activation rows per pass.
int32_t lp_chunk_nodes(const grf_graph* g, int32_t L) {
  int64_t c = ((int64_t)1 << 20) / std::max<int32_t>(g->nv, 1);
  if (c < 1) c = 1;
  return (int32_t)std::min<int64_t>(c, L);
}

// Inference activations of `nodes` nodes: two alternating hidden and two
// alternating concatenated-input buffers suffice for a forward pass.
void carve_lp_infer(Carve& c, const grf_graph* g, int32_t nodes, LpActs* a) {
  const size_t M = (size_t)nodes * g->nv;
  a->X0 = c.take<__nv_bfloat16>(M * 16);
  float* h0 = c.take<float>(M * 64);
  float* h1 = c.take<float>(M * 64);
  __nv_bfloat16* x0 = c.take<__nv_bfloat16>(M * 128);
  __nv_bfloat16* x1 = c.take<__nv_bfloat16>(M * 128);
  a->H[0] = h0; a->H[1] = h1; a->H[2] = h0; a->H[3] = h1;
  a->Xc[0] = x0; a->Xc[1] = x1; a->Xc[2] = x0;
  a->s = c.take<float>(M);
  a->al = c.take<float>(M);
  a->be = c.take<float>(M);
  a->es = nullptr;
  a->n = nullptr;
}

// The batched PCG's FP32-pair state (mixed precision): the blocks as pairs
// and the iterate and scaled right-hand side, hi and lo, shaped as r.
void carve_pairs(Carve& c, size_t Ls, size_t Sv, size_t V, size_t E, size_t tsize, ApplyWs* w) {
  w->dpair = w->opair = nullptr;
  w->xh = w->xl = w->gh = w->gl = nullptr;
  if (tsize != 4) return;
  w->dpair = c.take<float2>(Ls * V);
  w->opair = c.take<float2>(Ls * 2 * E);
  w->xh = c.take<float>(Ls * Sv * V);
  w->xl = c.take<float>(Ls * Sv * V);
  w->gh = c.take<float>(Ls * Sv * V);
  w->gl = c.take<float>(Ls * Sv * V);
}

void carve_apply(Carve& c, const grf_graph* g, int32_t L, int64_t S, size_t tsize, ApplyWs* w,
                 int precond = GRF_PRECOND_JACOBI, bool spectral = false, bool umma = false) {
  const size_t Ls = (size_t)L, E = (size_t)g->ne, V = (size_t)g->nv, Ss = (size_t)S;
  const size_t nsg = (Ss + recover_sample_group() - 1) / recover_sample_group();
  w->alpha = c.take<double>(Ls);
  w->gamma = c.take<double>(Ls);
  w->weight = c.take<double>(Ls);
  w->saa = c.take<double>(Ls * E);
  w->sab = c.take<double>(Ls * E);
  w->diag = c.take<double>(Ls * V);
  w->offv = c.take<double>(Ls * 2 * E);
  w->gvec = c.take<double>(Ls * Ss * V);
  w->x = c.take<double>(Ls * Ss * V);
  // FP32: samples padded to the batched PCG's groups of 8
  const size_t Sv = tsize == 4 ? (size_t)pcg_batch_padded_samples(S) : Ss;
  w->r = c.take<char>(Ls * Sv * V * tsize);
  w->p = c.take<char>(Ls * Sv * V * tsize);
  w->q = c.take<char>(Ls * Sv * V * tsize);
  w->d = c.take<char>(Ls * Sv * V * tsize);
  w->lpa = LpActs{};
  w->lp_chunk = 0;
  w->y = nullptr;
  w->pre_c = w->pre_n = nullptr;
  if (precond != GRF_PRECOND_JACOBI) {
    w->pre_c = c.take<char>(Ls * V * tsize);
    w->pre_n = c.take<char>(Ls * 2 * E * tsize);
  }
  if (precond == GRF_PRECOND_LEARNED) {
    w->y = c.take<char>(Ls * Ss * V * tsize);
    w->lp_chunk = lp_chunk_nodes(g, L);
    carve_lp_infer(c, g, w->lp_chunk, &w->lpa);
  }
  w->dscale = c.take<char>(Ls * V * tsize);
  w->offv_t = tsize == 4 ? c.take<char>(Ls * 2 * E * 4) : nullptr;
  carve_pairs(c, Ls, Sv, V, E, tsize, w);
  // scratch of the sequential recovery, only for edges longer than every bin
  const size_t ni_long = g->long_edges(tsize == 8) > 0 ? (size_t)g->ni : 0;
  w->acc = c.take<double>(ni_long * Ss);
  w->yscr = c.take<char>(ni_long * Ss * tsize);
  w->rpscr = c.take<char>(ni_long * nsg * tsize);
  w->prm = c.take<char>(Ls * E * 4 * tsize);
  w->xw = c.take<char>(Ls * Ss * V * tsize);
  w->bhat = spectral && tsize == 4 ? c.take<float>((size_t)g->ni * Ss) : nullptr;
  w->ends = spectral && umma && tsize == 4 ? c.take<float>(2 * E * Ss * Ls) : nullptr;
  w->nshift = c.take<float>(Ls);
  w->nwgam = c.take<float>(Ls);
  w->iters = c.take<int32_t>(Ls * Ss);
  w->status = c.take<PcgStatus>(1);
}

// Per-call statistics, kernel-launch count and (optional) CUDA-event phase timing.
struct RunStats {
  int64_t nodes = 0, systems = 0, iters_total = 0;
  int32_t iters_max = 0, unconverged = 0, numeric = 0, launches = 0, fallback = 0, timeouts = 0;
  bool timing = false;
  uint32_t mask = 0xFFu;  // the phases timed
  // graph capture: status words are copied to pinned host slots, no syncs
  bool capturing = false;
  PcgStatus* h_status = nullptr;
  int stage_idx = 0;
  std::vector<PhaseSpan> spans;
  cudaEvent_t open = nullptr;
  double phase_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};

  // Under stream capture an event record becomes a node of the graph (an
  // external event record), so each replay records the event again.
  void record(cudaEvent_t e, cudaStream_t st) const {
    if (capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
  }
  void begin(int phase, cudaStream_t st) {
    if (!timing || !((mask >> phase) & 1u)) return;
    cudaEventCreate(&open);
    record(open, st);
  }
  void end(int phase, cudaStream_t st) {
    if (!timing || !open || !((mask >> phase) & 1u)) return;
    cudaEvent_t b;
    cudaEventCreate(&b);
    record(b, st);
    spans.push_back({phase, open, b});
    open = nullptr;
  }
  // after the stream has been synchronised
  void settle() {
    for (auto& s : spans) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, s.a, s.b) == cudaSuccess) phase_ms[s.phase] += ms;
      cudaEventDestroy(s.a);
      cudaEventDestroy(s.b);
    }
    spans.clear();
  }
  ~RunStats() { settle(); }
};

DevNodes dev_nodes(const ApplyWs& w, int32_t L) {
  DevNodes d;
  d.L = L;
  d.alpha = w.alpha;
  d.gamma = w.gamma;
  d.weight = w.weight;
  d.shift = w.nshift;
  d.wgam = w.nwgam;
  return d;
}

int upload_nodes(const HostNodes& h, const ApplyWs& w, cudaStream_t st) {
  const size_t b = sizeof(double) * h.alpha.size();
  CUDA_TRY(cudaMemcpyAsync(w.alpha, h.alpha.data(), b, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(w.gamma, h.gamma.data(), b, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(w.weight, h.weight.data(), b, cudaMemcpyHostToDevice, st));
  return GRF_OK;
}

void add_status(const PcgStatus& h, RunStats* rs) {
  rs->iters_total += (int64_t)h.iters_total;
  if (h.iters_max > rs->iters_max) rs->iters_max = h.iters_max;
  rs->unconverged += h.n_unconverged;
  rs->numeric += h.numeric_flag;
  rs->fallback += h.n_fallback;
  rs->timeouts += h.device_timeout;
}

int collect(const ApplyWs& w, cudaStream_t st, int32_t L, int64_t S, RunStats* rs) {
  if (rs->capturing) {
    CUDA_TRY(cudaMemcpyAsync(rs->h_status + rs->stage_idx, w.status, sizeof(PcgStatus),
                             cudaMemcpyDeviceToHost, st));
    rs->stage_idx++;
    rs->nodes += L;
    rs->systems += (int64_t)L * S;
    return GRF_OK;
  }
  PcgStatus h{};
  CUDA_TRY(cudaMemcpyAsync(&h, w.status, sizeof h, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  rs->settle();
  rs->nodes += L;
  rs->systems += (int64_t)L * S;
  add_status(h, rs);
  return GRF_OK;
}

// The side stream on which the Schur blocks run beside the condensation.
int ensure_side(grf_graph* g) {
  if (g->side_stream) return GRF_OK;
  CUDA_TRY(cudaStreamCreateWithFlags(&g->side_stream, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
  return GRF_OK;
}

// Schur blocks + condensation + PCG for the nodes already uploaded to w.
template <typename T>
int vertex_phase(grf_graph* g, const ApplyWs& w, int32_t L, double kappa2, int64_t S,
                 const T* b, double* gvec, double* xv, const Opts& o, cudaStream_t st,
                 RunStats* rs, bool* xw_ready = nullptr) {
  const DevNodes nd = dev_nodes(w, L);
  CUDA_TRY(cudaMemsetAsync(w.status, 0, sizeof(PcgStatus), st));
  // the Thomas sweep constants are needed only where an edge is left to Thomas
  SweepParams<T>* prm = (SweepParams<T>*)w.prm;
  if (sizeof(T) == 4 && o.spectral && w.bhat && g->thomas_rest() == 0) prm = nullptr;
  // Without sweep constants nothing before the PCG reads the Schur blocks:
  // they run on a side stream beside the condensation (FP64-bound kernels
  // beside tensor-core and streaming ones) and the PCG waits for them.
  if (!prm && !rs->capturing) GRF_TRY(ensure_side(g));
  const bool side = !prm && g->side_stream;
  cudaStream_t sst = side ? g->side_stream : st;
  if (side) {
    CUDA_TRY(cudaEventRecord(g->ev_fork, st));
    CUDA_TRY(cudaStreamWaitEvent(sst, g->ev_fork, 0));
  }
  rs->begin(1, sst);
  rs->launches += launch_schur<T>(g->d, nd, kappa2, w.saa, w.sab, w.diag, w.offv, prm,
                                  (T*)w.dscale, (T*)w.offv_t, sst, o.consistent, w.dpair,
                                  w.opair);
  rs->end(1, sst);
  if (side) CUDA_TRY(cudaEventRecord(g->ev_join, sst));
  const int pre_kind = (sizeof(T) == 4 && o.precond == GRF_PRECOND_LEARNED)
                           ? kPreLearned
                           : (o.precond == GRF_PRECOND_NEUMANN ? kPreNeumann : kPreJacobi);
  bool g32 = false;  // g given to the PCG in FP32 (see below)
  rs->begin(2, st);
  if (sizeof(T) == 4) {
    // FP32: the tridiagonal edges (all of them, or those the spectral path
    // leaves over), short ones by segments and long ones by nodes, and the
    // spectral bins
    const bool spec = o.spectral && w.bhat;
    const int p = spec ? 2 : 0;
    if (spec) {
      launch_node_consts(nd, kappa2, w.nshift, w.nwgam, st);
      rs->launches += 1;
    }
    const int32_t head = bins_before(g, p, node_bin0(g, p, o, L));
    const int32_t tail = bins_total(g, p) - head;
    if (o.consistent && !(spec && umma_ready(g, o, S, L))) {
      if (side) cudaStreamWaitEvent(st, g->ev_join, 0);
      return fail(GRF_ENOTSUP, "the consistent mass needs the tensor-core sine transforms");
    }
    const bool umma = spec && umma_ready(g, o, S, L);
    // tensor-core path with the per-edge end-value buffer: its gather writes
    // g = b_v + (end values) for every node and sample, so it runs first and
    // the tridiagonal edges then add into it
    const bool gather_init = umma && w.ends;
    // When every edge with interior nodes is on the tensor-core path and the
    // batched PCG will run, the gather writes g in FP32 straight into that
    // PCG's layout (the end values and the noise are FP32 already)
    g32 = gather_init && head == 0 && tail == 0 && w.gh &&
          pcg_batch_selected(g->d, o.pcg_layout, pre_kind);
    if (umma) {
      rs->launches += launch_dst_gemm<false, float>(g->d, g->dst.dev, S, (const float*)b, w.bhat,
                                                    w.status, g->n_sm, st);
      if (!gather_init)
        rs->launches += launch_condense<T>(g->d, nd, kappa2, S, b, gvec, st, g->d_bin_edges[p], 0);
      rs->launches += launch_spec_ends_umma(g->d, nd, S, g->d_spec_edges, g->spec_count,
                                            g->n_spec_bins, w.bhat, gvec, w.ends,
                                            (const float*)b, o.consistent, w.status, g->n_sm,
                                            st, g32 ? w.gh : nullptr);
    }
    rs->launches += launch_condense<T>(g->d, nd, kappa2, S, b, gvec, st, g->d_bin_edges[p], head,
                                       !umma);
    if (tail > 0 && !prm) {
      if (side) cudaStreamWaitEvent(st, g->ev_join, 0);
      return fail(GRF_EINVAL, "node-parallel condensation of %d edges without sweep constants",
                  (int)tail);
    }
    if (tail > 0)
      rs->launches += launch_condense_nodes(g->d, L, S, (const float*)b,
                                            (const SweepParams<float>*)prm,
                                            g->d_bin_edges[p] + head, tail, gvec, st);
    if (!umma && spec && o.spec_tc)
      rs->launches += launch_spec_condense_mma(g->d, nd, S, (const float*)b, g->d_spec_edges,
                                               g->spec_count, w.bhat, gvec, st);
    else if (!umma && spec)
      rs->launches += launch_spec_condense(g->d, nd, kappa2, S, (const float*)b, g->d_spec_edges,
                                           g->spec_count, w.bhat, gvec, st);
  } else {
    rs->launches += launch_condense<T>(g->d, nd, kappa2, S, b, gvec, st);
  }
  rs->end(2, st);
  if (side) CUDA_TRY(cudaStreamWaitEvent(st, g->ev_join, 0));
  // FP64 PCG uses the FP64 blocks; the FP32 solve their scaled FP32 copy
  const T* offv_t = sizeof(T) == 8 ? (const T*)w.offv : (const T*)w.offv_t;
  const bool learned = sizeof(T) == 4 && o.precond == GRF_PRECOND_LEARNED;
  const bool neumann = o.precond == GRF_PRECOND_NEUMANN;
  if ((learned || neumann) && !w.pre_c)
    return fail(GRF_ENOTSUP, "this entry point has no workspace for preconditioner %d",
                o.precond);
  if (neumann) {
    launch_nn_coeffs<T>(g->d, L, w.saa, w.sab, w.diag, sizeof(T) == 4, (T*)w.pre_c,
                        (T*)w.pre_n, st);
    rs->launches += 1;
  }
  if (learned) {
    if (!g->lm.ready || w.lp_chunk < 1 || L > kRamp)
      return fail(GRF_EINVAL, "learned preconditioner not set up for this call");
    rs->begin(6, st);
    const int64_t ne2 = 2 * (int64_t)g->ne;
    for (int32_t l0 = 0; l0 < L; l0 += w.lp_chunk) {
      LpActs a = w.lpa;
      a.es = (float*)w.pre_c + (int64_t)l0 * g->nv;
      a.n = (float*)w.pre_n + (int64_t)l0 * ne2;
      const int32_t nb = std::min(w.lp_chunk, L - l0);
      rs->launches += lp_forward(g->d, nb, g->lm.ramp + l0, (const float*)w.offv_t, w.alpha,
                                 w.gamma, g->lm.P, g->lm.wb, a, st);
    }
    rs->end(6, st);
  }
  rs->begin(3, st);
  const int pre = learned ? kPreLearned : (neumann ? kPreNeumann : kPreJacobi);
  // with g in FP32 (the tensor-core sampler path) the PCG also hands the
  // recovery its weighted values w_l u^(l) directly
  const bool xw_out = g32 && w.xw && xw_ready;
  const PcgPairs pairs{w.dpair, w.opair, w.xh, w.xl, w.gh, w.gl, g32,
                       xw_out ? (float*)w.xw : nullptr, w.weight, xv};
  if (xw_ready) *xw_ready = xw_out;
  launch_pcg<T>(g->d, g->d_order, g->d_ell, L, S, w.diag, w.offv, (const T*)w.dscale, offv_t, pre,
                (const T*)w.pre_c, (const T*)w.pre_n, gvec, xv, (T*)w.d, (T*)w.r, (T*)w.p,
                (T*)w.q, (T*)w.y, o.rtol, o.max_iter, w.iters, w.status, o.pcg_layout, st,
                w.dpair ? &pairs : nullptr);
  rs->end(3, st);
  rs->launches += xw_out ? 2 : 1;  // the PCG (and its weighted-output pass)
  CUDA_TRY(cudaGetLastError());
  return GRF_OK;
}

// out = sum_l w_l A_l^{-1} b with b sample-minor [n][S] in precision T.
// nodes_dev (optional): alpha | gamma | weight already on the device.
template <typename T, typename OutT>
int dd_apply(grf_graph* g, const HostNodes& hn, double kappa, int64_t S, const T* b, OutT* out,
             const Opts& o, cudaStream_t st, void* ws_tail, RunStats* rs,
             const double* nodes_dev = nullptr) {
  Carve c(ws_tail);
  ApplyWs w;
  carve_apply(c, g, hn.L(), S, sizeof(T), &w, o.precond, o.spectral, o.spec_umma);
  const double k2 = kappa * kappa;
  if (nodes_dev) {
    w.alpha = const_cast<double*>(nodes_dev);
    w.gamma = const_cast<double*>(nodes_dev) + hn.L();
    w.weight = const_cast<double*>(nodes_dev) + 2 * hn.L();
  } else {
    GRF_TRY(upload_nodes(hn, w, st));
  }
  bool xw_ready = false;  // the PCG wrote the recovery's weighted values
  GRF_TRY(vertex_phase<T>(g, w, hn.L(), k2, S, b, w.gvec, w.x, o, st, rs, &xw_ready));
  const bool spec = sizeof(T) == 4 && o.spectral;
  const int p = sizeof(T) == 8 ? 1 : (spec ? 2 : 0);
  // FP32: bins from i0 on (and the edges beyond every bin) by the node sweeps
  const int i0 = sizeof(T) == 4 ? node_bin0(g, p, o, hn.L()) : g->n_bins[p] + 1;
  int32_t counts[kMaxBins + 1];
  for (int i = 0; i <= g->n_bins[p]; ++i) counts[i] = i < i0 ? g->bin_count[p][i] : 0;
  const int32_t head = bins_before(g, p, i0), tail = bins_total(g, p) - head;
  rs->begin(4, st);
  rs->launches += launch_recover<T, OutT>(g->d, dev_nodes(w, hn.L()), k2, S, b, w.x, out,
                                          (const SweepParams<T>*)w.prm, (T*)w.xw,
                                          g->d_bin_edges[p], counts, g->n_bins[p], w.acc,
                                          (T*)w.yscr, (T*)w.rpscr, o.recover_sg, st, xw_ready);
  if (sizeof(T) == 4 && tail > 0)
    rs->launches += launch_recover_nodes<OutT>(
        g->d, hn.L(), S, (const float*)b, (const SweepParams<float>*)w.prm, (const float*)w.xw,
        g->d_bin_edges[p] + head, tail, out, st);
  if (spec && umma_ready(g, o, S, hn.L())) {
    rs->launches += launch_spec_coef_umma(g->d, dev_nodes(w, hn.L()), S, g->d_spec_edges,
                                          g->spec_count, g->n_spec_bins, w.bhat,
                                          (const float*)w.xw, o.consistent, w.status, g->n_sm,
                                          st);
    rs->launches += launch_dst_gemm<true, OutT>(g->d, g->dst.dev, S, w.bhat, out, w.status,
                                                g->n_sm, st);
  } else if (spec) {
    rs->launches += launch_spec_recover<OutT>(g->d, dev_nodes(w, hn.L()), k2, S, g->d_spec_edges,
                                              g->spec_count, w.bhat, (const float*)w.xw, out, st);
  }
  rs->end(4, st);
  CUDA_TRY(cudaGetLastError());
  return collect(w, st, hn.L(), S, rs);
}

size_t apply_bytes(const grf_graph* g, int32_t L, int64_t S, size_t tsize, const Opts& o) {
  Carve c(nullptr);
  ApplyWs w;
  carve_apply(c, g, L, S, tsize, &w, o.precond, o.spectral, o.spec_umma);
  return c.off;
}

int finish(const RunStats& rs, grf_graph* g, grf_stats* stats) {
  if (stats) {
    stats->n_dofs = g->n;
    stats->n_nodes = rs.nodes;
    stats->n_systems = rs.systems;
    stats->pcg_iters_total = rs.iters_total;
    stats->pcg_iters_max = rs.iters_max;
    stats->n_unconverged = rs.unconverged;
    stats->numeric_flag = rs.numeric;
    stats->kernel_launches = rs.launches;
    stats->n_precond_fallback = rs.fallback;
    stats->reserved = 0;
    for (int i = 0; i < 8; ++i) stats->phase_ms[i] = rs.phase_ms[i];
  }
  if (rs.timeouts)
    return fail(GRF_ECUDA, "%d tensor-core kernels gave up waiting for their MMAs", rs.timeouts);
  if (rs.numeric) return fail(GRF_ENUMERIC, "NaN/Inf or non-positive p.Sp in %d PCG systems", rs.numeric);
  if (rs.unconverged)
    return fail(GRF_ENOCONV, "%d PCG systems did not converge", rs.unconverged);
  return GRF_OK;
}

int check_params(double kappa, double beta, double k_step) {
  if (!(kappa > 0) || !std::isfinite(kappa)) return fail(GRF_EINVAL, "kappa must be > 0");
  if (!(beta > 0) || !std::isfinite(beta) || beta > 64) return fail(GRF_EINVAL, "beta must be in (0, 64]");
  if (!(k_step > 0) || !std::isfinite(k_step)) return fail(GRF_EINVAL, "k_step must be > 0");
  return GRF_OK;
}

// Stages: the fractional part (or the first stiffness solve) then the integer powers.
void plan(double beta, double k_step, std::vector<HostNodes>* stages) {
  const double n_int = std::floor(beta);
  const double f = beta - n_int;
  if (f > 1e-12) {
    stages->push_back(quadrature_nodes(f, k_step));
    for (int i = 0; i < (int)n_int; ++i) stages->push_back(stiffness_node());
  } else {
    for (int i = 0; i < (int)n_int; ++i) stages->push_back(stiffness_node());
  }
}

size_t sample_ws_bytes(const grf_graph* g, const std::vector<HostNodes>& stages, int64_t S,
                       size_t tsize, const Opts& o) {
  size_t need = align_up((size_t)g->n * S * tsize);
  size_t tail = 0;
  for (auto& s : stages) tail = std::max(tail, apply_bytes(g, s.L(), S, tsize, o));
  if (stages.size() > 1) need += align_up((size_t)g->n * S * sizeof(double));
  if (o.consistent) need += align_up((size_t)g->nv * S * sizeof(float));  // vertex noise
  return need + tail;
}

// Enqueues one whole sample call on st (workspace already sized). With
// seed_dev / nodes_dev the seed and the node arrays come from device memory
// (graph capture); otherwise they are passed and uploaded here.
template <typename T, typename OutT>
int enqueue_sample(grf_graph* g, const std::vector<HostNodes>& stages, double kappa,
                   uint64_t seed, int64_t S, OutT* out, const Opts& o, cudaStream_t st,
                   RunStats* rs, const uint64_t* seed_dev = nullptr,
                   const std::vector<const double*>* nodes_dev = nullptr) {
  const bool multi = stages.size() > 1;
  Carve c(g->ws);
  T* b = c.take<T>((size_t)g->n * S);
  double* tmp = multi ? c.take<double>((size_t)g->n * S) : nullptr;
  float* wv = o.consistent ? c.take<float>((size_t)g->nv * S) : nullptr;
  void* ws_tail = g->ws ? (char*)g->ws + c.off : nullptr;
  rs->begin(0, st);
  if (sizeof(T) == 4 && o.consistent) {
    // W = R xi of the consistent mass: unit-mass normals, then the factor
    launch_noise_minor<float>(g->d, seed, S, (float*)b, st, seed_dev, g->cons.ones);
    rs->launches += launch_cons_noise(g->d, S, (float*)b, wv, g->cons.rp, g->cons.rc,
                                      g->cons.rv, g->n_sm, st);
  } else {
    launch_noise_minor<T>(g->d, seed, S, b, st, seed_dev, g->d_sqrt_ml_f);
  }
  rs->end(0, st);
  rs->launches += 1;
  CUDA_TRY(cudaGetLastError());
  for (size_t i = 0; i < stages.size(); ++i) {
    const bool last = i + 1 == stages.size();
    const double* nd = nodes_dev ? (*nodes_dev)[i] : nullptr;
    if (i > 0) {
      rs->begin(5, st);
      launch_to_minor<T>(g->d, S, tmp, b, true, st);
      rs->end(5, st);
      rs->launches += 1;
    }
    if (last) {
      GRF_TRY((dd_apply<T, OutT>(g, stages[i], kappa, S, b, out, o, st, ws_tail, rs, nd)));
    } else {
      GRF_TRY((dd_apply<T, double>(g, stages[i], kappa, S, b, tmp, o, st, ws_tail, rs, nd)));
    }
  }
  return GRF_OK;
}

template <typename T, typename OutT>
int sample_impl(grf_graph* g, double kappa, double beta, double k_step, uint64_t seed, int64_t S,
                OutT* out, const Opts& o, cudaStream_t st, RunStats* rs) {
  std::vector<HostNodes> stages;
  plan(beta, k_step, &stages);
  GRF_TRY(check_consistent(g, o, beta, S));
  GRF_TRY(check_fp32_range(g, o, kappa, stages));
  GRF_TRY(ensure_ws(g, sample_ws_bytes(g, stages, S, sizeof(T), o)));
  if (o.spec_umma) GRF_TRY(ensure_dst_plan(g, S));
  if (o.consistent) GRF_TRY(ensure_cons_plan(g));
  return enqueue_sample<T, OutT>(g, stages, kappa, seed, S, out, o, st, rs);
}

// The same call through a captured CUDA graph: captured once per configuration
// (on an internal stream), then replayed on the caller's stream with the seed
// copied in from pinned memory. Iteration statistics come back through pinned
// status slots. With phase timing the phase events are captured as event
// record nodes (a separate capture from the untimed one), and every replay
// adds their elapsed times to the call's phase_ms.
template <typename T, typename OutT>
int sample_graph_impl(grf_graph* g, double kappa, double beta, double k_step, uint64_t seed,
                      int64_t S, OutT* out, const Opts& o, cudaStream_t st, RunStats* rs) {
  std::vector<HostNodes> stages;
  plan(beta, k_step, &stages);
  GRF_TRY(check_consistent(g, o, beta, S));
  GRF_TRY(check_fp32_range(g, o, kappa, stages));
  GRF_TRY(ensure_ws(g, sample_ws_bytes(g, stages, S, sizeof(T), o)));
  if (o.spec_umma) GRF_TRY(ensure_dst_plan(g, S));
  if (o.consistent) GRF_TRY(ensure_cons_plan(g));
  auto& gc = g->gc;
  const bool hit = gc.valid && gc.precision == o.precision && gc.out_dtype == o.out_dtype &&
                   gc.precond == o.precond && gc.spectral == o.spectral && gc.sweep == o.sweep &&
                   gc.spec_tc == o.spec_tc && gc.spec_umma == o.spec_umma &&
                   gc.consistent == o.consistent &&
                   gc.timing == o.timing &&
                   gc.phase_mask == (o.timing ? o.phase_mask : 0u) &&
                   gc.pcg_layout == o.pcg_layout && gc.recover_sg == o.recover_sg &&
                   gc.max_iter == o.max_iter && gc.rtol == o.rtol && gc.kappa == kappa &&
                   gc.beta == beta && gc.k == k_step && gc.S == S && gc.out == (void*)out &&
                   gc.ws == g->ws;
  if (!hit) {
    g->drop_graph();
    size_t nd_count = 1;
    for (auto& s : stages) nd_count += 3 * (size_t)s.L();
    CUDA_TRY(cudaMalloc(&gc.nodes_dev, nd_count * sizeof(double)));
    std::vector<const double*> ptrs;
    size_t off = 0;
    for (auto& s : stages) {
      const size_t L = s.L();
      CUDA_TRY(cudaMemcpy(gc.nodes_dev + off, s.alpha.data(), L * 8, cudaMemcpyHostToDevice));
      CUDA_TRY(cudaMemcpy(gc.nodes_dev + off + L, s.gamma.data(), L * 8, cudaMemcpyHostToDevice));
      CUDA_TRY(
          cudaMemcpy(gc.nodes_dev + off + 2 * L, s.weight.data(), L * 8, cudaMemcpyHostToDevice));
      ptrs.push_back(gc.nodes_dev + off);
      off += 3 * L;
    }
    gc.d_seed = reinterpret_cast<uint64_t*>(gc.nodes_dev + off);
    if (!gc.h_seed) CUDA_TRY(cudaMallocHost(&gc.h_seed, sizeof(uint64_t)));
    if (gc.h_status_cap < (int)stages.size()) {
      if (gc.h_status) CUDA_TRY(cudaFreeHost(gc.h_status));
      gc.h_status = nullptr;
      CUDA_TRY(cudaMallocHost(&gc.h_status, sizeof(PcgStatus) * stages.size()));
      gc.h_status_cap = (int)stages.size();
    }
    if (!g->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    GRF_TRY(ensure_side(g));
    RunStats cap;
    cap.capturing = true;
    cap.timing = o.timing;
    cap.mask = o.phase_mask;
    cap.h_status = gc.h_status;
    CUDA_TRY(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed));
    const int r = enqueue_sample<T, OutT>(g, stages, kappa, 0, S, out, o, g->cap_stream, &cap,
                                          gc.d_seed, &ptrs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(g->cap_stream, &graph);
    if (r != GRF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return r;
    }
    if (ec != cudaSuccess) return fail(GRF_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
    const cudaError_t ei = cudaGraphInstantiate(&gc.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(GRF_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
    gc.spans = std::move(cap.spans);  // owned by the cache from here on
    cap.spans.clear();
    gc.stage_L.clear();
    for (auto& s : stages) gc.stage_L.push_back(s.L());
    gc.launches = cap.launches;
    gc.precision = o.precision;
    gc.precond = o.precond;
    gc.spectral = o.spectral;
    gc.spec_tc = o.spec_tc;
    gc.spec_umma = o.spec_umma;
    gc.consistent = o.consistent;
    gc.timing = o.timing;
    gc.phase_mask = o.timing ? o.phase_mask : 0u;
    gc.sweep = o.sweep;
    gc.out_dtype = o.out_dtype;
    gc.pcg_layout = o.pcg_layout;
    gc.recover_sg = o.recover_sg;
    gc.max_iter = o.max_iter;
    gc.rtol = o.rtol;
    gc.kappa = kappa;
    gc.beta = beta;
    gc.k = k_step;
    gc.S = S;
    gc.out = (void*)out;
    gc.ws = g->ws;
    gc.valid = true;
  }
  *gc.h_seed = seed;
  CUDA_TRY(cudaMemcpyAsync(gc.d_seed, gc.h_seed, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaGraphLaunch(gc.exec, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (const auto& sp : gc.spans) {  // this replay's phase events
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, sp.a, sp.b) == cudaSuccess) rs->phase_ms[sp.phase] += ms;
  }
  for (size_t i = 0; i < gc.stage_L.size(); ++i) {
    add_status(gc.h_status[i], rs);
    rs->nodes += gc.stage_L[i];
    rs->systems += (int64_t)gc.stage_L[i] * S;
  }
  rs->launches += gc.launches;
  return GRF_OK;
}

int check_graph(const grf_graph* g) {
  if (!g) return fail(GRF_EINVAL, "null graph");
  return GRF_OK;
}

}  // namespace

// Scratch of grf_vertex_solve_noalloc: one fixed device array that every GPU
// loading this library holds until the process exits. Host code must not pass
// this name to a kernel (on the host it is only a stand-in for the symbol);
// the device address comes from cudaGetSymbolAddress below.
static constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) unsigned char grf_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of grf_noalloc_scratch on device `dev` (which must be the
// current device), looked up once per device and cached.
int noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(GRF_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, grf_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(GRF_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                  cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return GRF_OK;
}

// The part of an apply workspace one vertex solve touches (no recovery buffers).
void carve_vertex_solve(Carve& c, const grf_graph* g, int64_t S, size_t tsize, ApplyWs* w, void** b) {
  const size_t E = (size_t)g->ne, V = (size_t)g->nv, Ss = (size_t)S;
  *b = c.take<char>((size_t)g->n * Ss * tsize);
  w->alpha = c.take<double>(1);
  w->gamma = c.take<double>(1);
  w->weight = c.take<double>(1);
  w->saa = c.take<double>(E);
  w->sab = c.take<double>(E);
  w->diag = c.take<double>(V);
  w->offv = c.take<double>(2 * E);
  const size_t Sv = tsize == 4 ? (size_t)pcg_batch_padded_samples(S) : Ss;
  w->r = c.take<char>(Sv * V * tsize);
  w->p = c.take<char>(Sv * V * tsize);
  w->q = c.take<char>(Sv * V * tsize);
  w->d = c.take<char>(Sv * V * tsize);
  w->y = nullptr;
  w->pre_c = w->pre_n = nullptr;
  w->dscale = c.take<char>(V * tsize);
  w->offv_t = tsize == 4 ? c.take<char>(2 * E * 4) : nullptr;
  carve_pairs(c, 1, Sv, V, E, tsize, w);
  w->iters = c.take<int32_t>(Ss);
  w->status = c.take<PcgStatus>(1);
  // sweep constants of the one node: launch_schur fills them and the
  // node-parallel condensation of the long FP32 edges reads them
  w->prm = c.take<char>(E * 4 * tsize);
  w->gvec = w->x = w->acc = nullptr;
  w->yscr = w->rpscr = nullptr;
  w->xw = nullptr;
  w->bhat = nullptr;
  w->ends = nullptr;
  w->nshift = w->nwgam = nullptr;
}

// ---- learned preconditioner: model storage, initialisation and helpers

int ensure_model(grf_graph* g) {
  GRF_TRY(ensure_device(g));
  LearnedModel& lm = g->lm;
  if (lm.blk) return GRF_OK;
  Carve dry(nullptr);
  for (int i = 0; i < 4; ++i) dry.take<float>(kParams);
  dry.take<__nv_bfloat16>(kWbf16);
  dry.take<__nv_bfloat16>(kWtbf16);
  dry.take<int32_t>(kRamp);
  void* blk = nullptr;
  CUDA_TRY(cudaMalloc(&blk, dry.off));
  lm.blk = blk;
  Carve c(blk);
  lm.P = c.take<float>(kParams);
  lm.G = c.take<float>(kParams);
  lm.m = c.take<float>(kParams);
  lm.v = c.take<float>(kParams);
  lm.wb = c.take<__nv_bfloat16>(kWbf16);
  lm.wt = c.take<__nv_bfloat16>(kWtbf16);
  lm.ramp = c.take<int32_t>(kRamp);
  CUDA_TRY(cudaMemset(blk, 0, dry.off));
  std::vector<int32_t> ramp(kRamp);
  for (int i = 0; i < kRamp; ++i) ramp[i] = i;
  CUDA_TRY(cudaMemcpy(lm.ramp, ramp.data(), sizeof(int32_t) * kRamp, cudaMemcpyHostToDevice));
  return GRF_OK;
}

// New FP32 weights: BF16 copies refreshed, optimiser state cleared.
int model_set(grf_graph* g, const float* host) {
  GRF_TRY(ensure_model(g));
  LearnedModel& lm = g->lm;
  CUDA_TRY(cudaMemcpy(lm.P, host, sizeof(float) * kParams, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemset(lm.G, 0, sizeof(float) * kParams));
  CUDA_TRY(cudaMemset(lm.m, 0, sizeof(float) * kParams));
  CUDA_TRY(cudaMemset(lm.v, 0, sizeof(float) * kParams));
  lp_weights_bf16(lm.P, lm.wb, lm.wt, nullptr);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaDeviceSynchronize());
  lm.step = 0;
  lm.ready = true;
  return GRF_OK;
}

// splitmix64 (Steele, Lea, Flood 2014) and Box-Muller normals for the host-side
// weight initialisation.
uint64_t splitmix64(uint64_t* s) {
  uint64_t z = (*s += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
double host_normal(uint64_t* s) {
  const double u1 = ((double)(splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((double)(splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

bool params_finite(const float* p) {
  for (int i = 0; i < kParams; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Full activations and gradients of a training pass over `nodes` nodes.
void carve_lp_train(Carve& c, const grf_graph* g, int32_t nodes, int pair_ctas, LpActs* a,
                    LpGrads* b) {
  const size_t M = (size_t)nodes * g->nv, ne2 = 2 * (size_t)g->ne;
  a->X0 = c.take<__nv_bfloat16>(M * 16);
  for (int i = 0; i <= kLayers; ++i) a->H[i] = c.take<float>(M * 64);
  for (int i = 0; i < kLayers; ++i) a->Xc[i] = c.take<__nv_bfloat16>(M * 128);
  a->s = c.take<float>(M);
  a->es = c.take<float>(M);
  a->al = c.take<float>(M);
  a->be = c.take<float>(M);
  a->n = c.take<float>((size_t)nodes * ne2);
  b->ds = c.take<float>(M);
  b->dn = c.take<float>((size_t)nodes * ne2);
  b->dH = c.take<float>(M * 64);
  b->dX = c.take<float>(M * 128);
  b->dA = c.take<__nv_bfloat16>(M * 64);
  b->max_pair_ctas = pair_ctas;
  b->scratch = c.take<float>((size_t)pair_ctas * 4 * g->nv);
}

// Per-node Schur data of a training or test pass (mixed-precision form).
struct LpNodes {
  double *alpha, *gamma, *weight, *saa, *sab, *diag, *offv;
  float *dscale, *offv_t;
};
void carve_lp_nodes(Carve& c, const grf_graph* g, int32_t L, LpNodes* n) {
  const size_t Ls = L, E = g->ne, V = g->nv;
  n->alpha = c.take<double>(Ls);
  n->gamma = c.take<double>(Ls);
  n->weight = c.take<double>(Ls);
  n->saa = c.take<double>(Ls * E);
  n->sab = c.take<double>(Ls * E);
  n->diag = c.take<double>(Ls * V);
  n->offv = c.take<double>(Ls * 2 * E);
  n->dscale = c.take<float>(Ls * V);
  n->offv_t = c.take<float>(Ls * 2 * E);
}
int lp_node_setup(grf_graph* g, const HostNodes& hn, double kappa, const LpNodes& n,
                  cudaStream_t st) {
  const size_t b = sizeof(double) * hn.alpha.size();
  CUDA_TRY(cudaMemcpyAsync(n.alpha, hn.alpha.data(), b, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(n.gamma, hn.gamma.data(), b, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(n.weight, hn.weight.data(), b, cudaMemcpyHostToDevice, st));
  DevNodes nd{hn.L(), n.alpha, n.gamma, n.weight};
  launch_schur<float>(g->d, nd, kappa * kappa, n.saa, n.sab, n.diag, n.offv, nullptr, n.dscale,
                      n.offv_t, st);
  CUDA_TRY(cudaGetLastError());
  return GRF_OK;
}

struct DeviceBlock {
  void* p = nullptr;
  ~DeviceBlock() {
    if (p) cudaFree(p);
  }
};

// Forward (and, with pairs, loss and gradient) of the network for one node.
int lp_single(grf_graph* g, double kappa, double alpha, double gamma, int64_t n_pairs,
              const float* R, const float* E, float* s_out, float* n_out, double* loss,
              float* grad, cudaStream_t st) {
  GRF_TRY(check_graph(g));
  if (!(kappa > 0) || !(alpha > 0) || !(gamma > 0) || !std::isfinite(alpha) ||
      !std::isfinite(gamma))
    return fail(GRF_EINVAL, "need kappa > 0, alpha > 0, gamma > 0");
  if (n_pairs < 0 || (n_pairs > 0 && (!R || !E))) return fail(GRF_EINVAL, "bad pairs");
  if (!g->lm.ready) return fail(GRF_EINVAL, "no preconditioner weights on this graph");
  GRF_TRY(ensure_device(g));
  const int pair_ctas = (int)std::max<int64_t>(1, std::min<int64_t>(n_pairs, 1024));
  const size_t V = g->nv, ne2 = 2 * (size_t)g->ne;
  HostNodes hn;
  hn.alpha = {alpha};
  hn.gamma = {gamma};
  hn.weight = {1.0};
  LpNodes nn;
  LpActs a;
  LpGrads b;
  float *dR = nullptr, *dE = nullptr, *G = nullptr, *dloss = nullptr;
  int32_t* pj = nullptr;
  DeviceBlock blk;
  for (int pass = 0; pass < 2; ++pass) {
    Carve c(pass ? blk.p : nullptr);
    carve_lp_nodes(c, g, 1, &nn);
    carve_lp_train(c, g, 1, pair_ctas, &a, &b);
    dR = c.take<float>((size_t)n_pairs * V);
    dE = c.take<float>((size_t)n_pairs * V);
    pj = c.take<int32_t>((size_t)n_pairs);
    G = c.take<float>(kParams);
    dloss = c.take<float>(1);
    if (!pass) CUDA_TRY(cudaMalloc(&blk.p, c.off));
  }
  GRF_TRY(lp_node_setup(g, hn, kappa, nn, st));
  lp_forward(g->d, 1, g->lm.ramp, nn.offv_t, nn.alpha, nn.gamma, g->lm.P, g->lm.wb, a, st);
  CUDA_TRY(cudaGetLastError());
  if (n_pairs > 0) {
    CUDA_TRY(cudaMemcpyAsync(dR, R, sizeof(float) * n_pairs * V, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(dE, E, sizeof(float) * n_pairs * V, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(pj, 0, sizeof(int32_t) * n_pairs, st));
    CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(float) * kParams, st));
    CUDA_TRY(cudaMemsetAsync(dloss, 0, sizeof(float), st));
    lp_backward(g->d, 1, g->lm.ramp, nn.offv_t, g->lm.P, g->lm.wt, a, n_pairs, pj, nullptr, dR,
                dE, (float)(1.0 / (double)n_pairs), b, G, dloss, st);
    CUDA_TRY(cudaGetLastError());
  }
  if (s_out) CUDA_TRY(cudaMemcpyAsync(s_out, a.s, sizeof(float) * V, cudaMemcpyDeviceToHost, st));
  if (n_out)
    CUDA_TRY(cudaMemcpyAsync(n_out, a.n, sizeof(float) * ne2, cudaMemcpyDeviceToHost, st));
  float hl = 0.f;
  if (n_pairs > 0) {
    if (grad) CUDA_TRY(cudaMemcpyAsync(grad, G, sizeof(float) * kParams, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&hl, dloss, sizeof(float), cudaMemcpyDeviceToHost, st));
  } else if (grad) {
    std::memset(grad, 0, sizeof(float) * kParams);
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  if (loss) *loss = hl;
  return GRF_OK;
}

struct LpFileHeader {
  char magic[8];
  int32_t version, n_params, n_features, width, layers, feature_set;
  int32_t reserved[4];
};
static_assert(sizeof(LpFileHeader) == 48, "weights file header is 48 bytes");

}  // namespace

extern "C" {

const char* grf_last_error(void) { return g_last_error.c_str(); }

int grf_precond_init(grf_graph* g, uint64_t seed) {
  GRF_TRY(check_graph(g));
  std::vector<float> p(kParams, 0.f);
  uint64_t st = seed ^ 0x6c8e9cf570932bd5ULL;
  for (int i = 0; i < kFeat * 64; ++i)
    p[kOffW0 + i] = (float)(host_normal(&st) * std::sqrt(2.0 / kFeat));
  for (int l = 1; l <= kLayers; ++l)
    for (int i = 0; i < 128 * 64; ++i)
      p[layer_w_off(l) + i] = (float)(host_normal(&st) * std::sqrt(2.0 / 128));
  return model_set(g, p.data());
}

int grf_precond_set(grf_graph* g, const float* params, int64_t n) {
  GRF_TRY(check_graph(g));
  if (!params || n != kParams)
    return fail(GRF_EINVAL, "need %d parameters (got %lld)", kParams, (long long)n);
  if (!params_finite(params)) return fail(GRF_EINVAL, "non-finite parameter");
  return model_set(g, params);
}

int grf_precond_get(const grf_graph* g, float* params, int64_t n) {
  GRF_TRY(check_graph(g));
  if (!params || n != kParams)
    return fail(GRF_EINVAL, "need room for %d parameters (got %lld)", kParams, (long long)n);
  if (!g->lm.ready) return fail(GRF_EINVAL, "no preconditioner weights on this graph");
  int cur = 0;
  CUDA_TRY(cudaGetDevice(&cur));
  if (cur != g->device) return fail(GRF_EINVAL, "graph lives on device %d", g->device);
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(params, g->lm.P, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
  return GRF_OK;
}

int grf_precond_save(const grf_graph* g, const char* path) {
  if (!path) return fail(GRF_EINVAL, "null path");
  std::vector<float> p(kParams);
  GRF_TRY(grf_precond_get(g, p.data(), kParams));
  LpFileHeader h{};
  std::memcpy(h.magic, "GRFLPBB1", 8);
  h.version = 1;
  h.n_params = kParams;
  h.n_features = kFeat;
  h.width = 64;
  h.layers = kLayers;
  h.feature_set = 1;
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(GRF_EINVAL, "cannot open %s for writing", path);
  const bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 &&
                  std::fwrite(p.data(), sizeof(float), kParams, f) == (size_t)kParams;
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed) return fail(GRF_EINVAL, "write to %s failed", path);
  return GRF_OK;
}

int grf_precond_load(grf_graph* g, const char* path) {
  GRF_TRY(check_graph(g));
  if (!path) return fail(GRF_EINVAL, "null path");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(GRF_EINVAL, "cannot open %s", path);
  LpFileHeader h{};
  std::vector<float> p(kParams);
  const bool ok = std::fread(&h, sizeof h, 1, f) == 1 &&
                  std::fread(p.data(), sizeof(float), kParams, f) == (size_t)kParams;
  char extra;
  const bool at_end = std::fread(&extra, 1, 1, f) == 0;
  std::fclose(f);
  if (!ok) return fail(GRF_EINVAL, "%s is too short for a weights file", path);
  if (std::memcmp(h.magic, "GRFLPBB1", 8) != 0 || h.version != 1 || h.n_params != kParams ||
      h.n_features != kFeat || h.width != 64 || h.layers != kLayers || h.feature_set != 1 ||
      h.reserved[0] || h.reserved[1] || h.reserved[2] || h.reserved[3] || !at_end)
    return fail(GRF_EINVAL, "%s is not a version-1 weights file of this network", path);
  if (!params_finite(p.data())) return fail(GRF_EINVAL, "%s holds non-finite weights", path);
  return model_set(g, p.data());
}

int grf_precond_forward(grf_graph* g, double kappa, double alpha, double gamma, float* s_out,
                        float* n_out, void* stream) {
  return lp_single(g, kappa, alpha, gamma, 0, nullptr, nullptr, s_out, n_out, nullptr, nullptr,
                   (cudaStream_t)stream);
}

int grf_precond_loss_grad(grf_graph* g, double kappa, double alpha, double gamma,
                          int64_t n_pairs, const float* R, const float* E, double* loss,
                          float* grad, void* stream) {
  if (n_pairs < 1) return fail(GRF_EINVAL, "need n_pairs >= 1");
  return lp_single(g, kappa, alpha, gamma, n_pairs, R, E, nullptr, nullptr, loss, grad,
                   (cudaStream_t)stream);
}

int grf_precond_train(grf_graph* g, double kappa, double beta, double k_step,
                      const grf_train_options* opts, float* loss_history, int64_t* n_pairs,
                      void* stream) {
  GRF_TRY(check_graph(g));
  GRF_TRY(check_params(kappa, beta, k_step));
  if (!g->lm.ready) return fail(GRF_EINVAL, "initialise or load the weights before training");
  grf_train_options o{};
  if (opts) o = *opts;
  const int epochs = o.epochs > 0 ? o.epochs : 40;
  const int nb = o.nodes_per_batch > 0 ? o.nodes_per_batch : 8;
  const int St = o.n_samples > 0 ? o.n_samples : 8;
  const int per = o.pairs_per_system > 0 ? o.pairs_per_system : 16;
  const int stride = o.record_stride > 0 ? o.record_stride : 2;
  const int max_iter = o.max_iter > 0 ? o.max_iter : 4000;
  const double rtol = o.rtol > 0 ? o.rtol : 1e-10;
  const float lr = (float)(o.lr > 0 ? o.lr : 1e-3);
  if (epochs > 100000 || St > 4096 || per > 4096 || nb > 4096)
    return fail(GRF_EINVAL, "training options out of range");
  GRF_TRY(ensure_device(g));
  cudaStream_t st = (cudaStream_t)stream;
  // training nodes: those of the sample call, each (alpha, gamma) once
  std::vector<HostNodes> stages;
  plan(beta, k_step, &stages);
  HostNodes hn;
  for (auto& sg : stages)
    for (int32_t i = 0; i < sg.L(); ++i) {
      bool seen = false;
      for (int32_t j = 0; j < hn.L(); ++j)
        seen = seen || (hn.alpha[j] == sg.alpha[i] && hn.gamma[j] == sg.gamma[i]);
      if (!seen) {
        hn.alpha.push_back(sg.alpha[i]);
        hn.gamma.push_back(sg.gamma[i]);
        hn.weight.push_back(1.0);
      }
    }
  const int32_t L = hn.L();
  if (L > kRamp) return fail(GRF_ENOTSUP, "too many quadrature nodes (%d)", L);
  const int32_t Lb = std::min<int32_t>(nb, L);
  const size_t V = g->nv, nsys = (size_t)L * St, nrec = nsys * per;
  const int rec_ctas = (int)std::min<size_t>(nsys, 304);
  // batches: every epoch a random order of the nodes, cut into groups of Lb
  std::vector<int32_t> order(L);
  uint64_t rs = o.seed ^ 0x243f6a8885a308d3ULL;
  struct Step {
    int64_t lnode_off, pair_off, npairs;
    int32_t nodes, epoch;
  };
  std::vector<Step> steps;
  std::vector<int32_t> lnode_all;
  const int pair_ctas = 1024;
  // phase 1: pairs
  LpNodes nn;
  float *b = nullptr, *R = nullptr, *E = nullptr;
  double *gvec = nullptr, *work = nullptr, *xrec = nullptr, *rinv = nullptr;
  int32_t* count = nullptr;
  DeviceBlock data;
  for (int pass = 0; pass < 2; ++pass) {
    Carve c(pass ? data.p : nullptr);
    carve_lp_nodes(c, g, L, &nn);
    b = c.take<float>((size_t)g->n * St);
    gvec = c.take<double>(nsys * V);
    work = c.take<double>((size_t)rec_ctas * 4 * V);
    xrec = c.take<double>((size_t)rec_ctas * per * V);
    R = c.take<float>(nrec * V);
    E = c.take<float>(nrec * V);
    rinv = c.take<double>(nrec);
    count = c.take<int32_t>(nsys);
    if (!pass) CUDA_TRY(cudaMalloc(&data.p, c.off));
  }
  GRF_TRY(lp_node_setup(g, hn, kappa, nn, st));
  DevNodes nd{L, nn.alpha, nn.gamma, nn.weight};
  launch_noise_minor<float>(g->d, o.seed, St, b, st, nullptr, g->d_sqrt_ml_f);
  launch_condense<float>(g->d, nd, kappa * kappa, St, b, gvec, st);
  lp_record_pairs(g->d, (int64_t)nsys, St, nn.diag, nn.offv, gvec, work, xrec, R, E, rinv, count,
                  per, stride, rtol, max_iter, rec_ctas, st);
  CUDA_TRY(cudaGetLastError());
  std::vector<int32_t> cnt(nsys);
  CUDA_TRY(cudaMemcpyAsync(cnt.data(), count, sizeof(int32_t) * nsys, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  // pair lists per node: slot = (l * St + s) * per + i
  std::vector<std::vector<int64_t>> node_slots(L);
  int64_t total_pairs = 0;
  for (int32_t l = 0; l < L; ++l)
    for (int s = 0; s < St; ++s) {
      const size_t sys = (size_t)l * St + s;
      for (int i = 0; i < cnt[sys] && i < per; ++i) node_slots[l].push_back((int64_t)sys * per + i);
      total_pairs += std::min(cnt[sys], per);
    }
  if (n_pairs) *n_pairs = total_pairs;
  std::vector<int32_t> pj_all;
  std::vector<int64_t> slot_all;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int32_t i = 0; i < L; ++i) order[i] = i;
    for (int32_t i = L - 1; i > 0; --i) {
      const int32_t j = (int32_t)(splitmix64(&rs) % (uint64_t)(i + 1));
      std::swap(order[i], order[j]);
    }
    for (int32_t i0 = 0; i0 < L; i0 += Lb) {
      Step s{(int64_t)lnode_all.size(), (int64_t)pj_all.size(), 0,
             std::min<int32_t>(Lb, L - i0), ep};
      for (int32_t j = 0; j < s.nodes; ++j) {
        const int32_t l = order[i0 + j];
        lnode_all.push_back(l);
        for (int64_t sl : node_slots[l]) {
          pj_all.push_back(j);
          slot_all.push_back(sl);
        }
      }
      s.npairs = (int64_t)pj_all.size() - s.pair_off;
      if (s.npairs > 0) steps.push_back(s);
    }
  }
  // phase 2: Adam steps
  LpActs a;
  LpGrads gr;
  int32_t *d_lnode = nullptr, *d_pj = nullptr;
  int64_t* d_slot = nullptr;
  float* d_loss = nullptr;
  DeviceBlock tb;
  for (int pass = 0; pass < 2; ++pass) {
    Carve c(pass ? tb.p : nullptr);
    carve_lp_train(c, g, Lb, pair_ctas, &a, &gr);
    d_lnode = c.take<int32_t>(std::max<size_t>(1, lnode_all.size()));
    d_pj = c.take<int32_t>(std::max<size_t>(1, pj_all.size()));
    d_slot = c.take<int64_t>(std::max<size_t>(1, slot_all.size()));
    d_loss = c.take<float>(std::max<size_t>(1, steps.size()));
    if (!pass) CUDA_TRY(cudaMalloc(&tb.p, c.off));
  }
  CUDA_TRY(cudaMemcpyAsync(d_lnode, lnode_all.data(), 4 * lnode_all.size(), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(d_pj, pj_all.data(), 4 * pj_all.size(), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(d_slot, slot_all.data(), 8 * slot_all.size(), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(d_loss, 0, sizeof(float) * std::max<size_t>(1, steps.size()), st));
  LearnedModel& lm = g->lm;
  CUDA_TRY(cudaMemsetAsync(lm.G, 0, sizeof(float) * kParams, st));
  for (size_t i = 0; i < steps.size(); ++i) {
    const Step& s = steps[i];
    lp_forward(g->d, s.nodes, d_lnode + s.lnode_off, nn.offv_t, nn.alpha, nn.gamma, lm.P, lm.wb,
               a, st);
    lp_backward(g->d, s.nodes, d_lnode + s.lnode_off, nn.offv_t, lm.P, lm.wt, a, s.npairs,
                d_pj + s.pair_off, d_slot + s.pair_off, R, E, (float)(1.0 / (double)s.npairs),
                gr, lm.G, d_loss + i, st);
    lp_adam(lm.P, lm.G, lm.m, lm.v, lr, ++lm.step, st);
    lp_weights_bf16(lm.P, lm.wb, lm.wt, st);
  }
  CUDA_TRY(cudaGetLastError());
  std::vector<float> hl(std::max<size_t>(1, steps.size()));
  CUDA_TRY(cudaMemcpyAsync(hl.data(), d_loss, sizeof(float) * hl.size(), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (loss_history) {
    std::vector<double> sum(epochs, 0.0);
    std::vector<int> n(epochs, 0);
    for (size_t i = 0; i < steps.size(); ++i) {
      sum[steps[i].epoch] += hl[i];
      n[steps[i].epoch]++;
    }
    for (int e = 0; e < epochs; ++e) loss_history[e] = n[e] ? (float)(sum[e] / n[e]) : 0.f;
  }
  std::vector<float> p(kParams);
  CUDA_TRY(cudaMemcpy(p.data(), lm.P, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
  if (!params_finite(p.data())) {
    lm.ready = false;
    return fail(GRF_ENUMERIC, "training diverged (non-finite weights); weights disabled");
  }
  return GRF_OK;
}

// Reverse Cuthill-McKee order of the kept vertices: a breadth-first search
// from a vertex of smallest degree in each component, the new neighbours of
// every vertex taken by increasing degree, the whole order reversed. Adjacent
// vertices end up in nearby slots, so the shared-memory PCG that stores its
// system in this order gathers neighbour rows from a narrow band.
static void rcm_order(grf_graph& g) {
  const int32_t nv = g.nv;
  std::vector<int32_t> deg(nv);
  for (int32_t v = 0; v < nv; ++v) deg[v] = g.vptr[v + 1] - g.vptr[v];
  const auto by_degree = [&deg](int32_t a, int32_t b) {
    return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
  };
  std::vector<int32_t> roots(nv);
  for (int32_t v = 0; v < nv; ++v) roots[v] = v;
  std::sort(roots.begin(), roots.end(), by_degree);
  std::vector<int32_t> order;
  order.reserve(nv);
  std::vector<char> seen(nv, 0);
  std::vector<int32_t> fresh;
  for (const int32_t r : roots) {
    if (seen[r]) continue;
    seen[r] = 1;
    size_t head = order.size();
    order.push_back(r);
    while (head < order.size()) {
      const int32_t v = order[head++];
      fresh.clear();
      for (int32_t k = g.vptr[v]; k < g.vptr[v + 1]; ++k) {
        const int32_t w = g.adj_nbr[k];
        if (!seen[w]) {
          seen[w] = 1;
          fresh.push_back(w);
        }
      }
      std::sort(fresh.begin(), fresh.end(), by_degree);
      order.insert(order.end(), fresh.begin(), fresh.end());
    }
  }
  std::reverse(order.begin(), order.end());
  std::vector<int32_t> slot(nv);
  for (int32_t i = 0; i < nv; ++i) slot[order[i]] = i;
  g.rperm = order;
  g.rvptr.assign(nv + 1, 0);
  for (int32_t i = 0; i < nv; ++i) g.rvptr[i + 1] = g.rvptr[i] + deg[order[i]];
  g.rnbr.resize(g.adj_nbr.size());
  g.rinc.resize(g.adj_nbr.size());
  for (int32_t i = 0; i < nv; ++i) {
    const int32_t v = order[i];
    for (int32_t j = 0; j < deg[v]; ++j) {
      const int32_t k = g.vptr[v] + j;
      g.rnbr[g.rvptr[i] + j] = slot[g.adj_nbr[k]];
      g.rinc[g.rvptr[i] + j] = k;
    }
  }
}

int grf_graph_create(int64_t n_vertices, int64_t n_edges, const int64_t* edge_u,
                     const int64_t* edge_v, const double* lengths, const int32_t* n_elems,
                     double h, grf_graph** out) {
  if (!out) return fail(GRF_EINVAL, "out is null");
  *out = nullptr;
  if (n_vertices < 1 || n_edges < 1) return fail(GRF_EINVAL, "need at least one vertex and edge");
  if (n_edges > (int64_t)1 << 29 || n_vertices > (int64_t)1 << 30)
    return fail(GRF_EINVAL, "graph too large");
  if (!edge_u || !edge_v || !lengths) return fail(GRF_EINVAL, "null edge arrays");
  if (!n_elems && !(h > 0 && std::isfinite(h))) return fail(GRF_EINVAL, "need n_elems or h > 0");
  grf_graph* g = new (std::nothrow) grf_graph();
  if (!g) return fail(GRF_ENOMEM, "host allocation failed");
  const int64_t E = n_edges;
  std::vector<int64_t> deg(n_vertices, 0);
  for (int64_t e = 0; e < E; ++e) {
    const int64_t a = edge_u[e], b = edge_v[e];
    if (a < 0 || a >= n_vertices || b < 0 || b >= n_vertices) {
      delete g;
      return fail(GRF_EINVAL, "edge %lld has an endpoint out of range", (long long)e);
    }
    if (a == b) {
      delete g;
      return fail(GRF_EINVAL, "edge %lld is a self-loop", (long long)e);
    }
    if (!(lengths[e] > 0) || !std::isfinite(lengths[e])) {
      delete g;
      return fail(GRF_EINVAL, "edge %lld has a non-positive or non-finite length", (long long)e);
    }
    deg[a]++;
    deg[b]++;
  }
  g->nv_in = n_vertices;
  g->vertex_map.assign(n_vertices, -1);
  int32_t nv = 0;
  for (int64_t v = 0; v < n_vertices; ++v)
    if (deg[v] > 0) g->vertex_map[v] = nv++;
  g->nv = nv;
  g->ne = (int32_t)E;
  g->eu.resize(E);
  g->ev.resize(E);
  g->nel.resize(E);
  g->he.resize(E);
  g->ioff.assign(E + 1, 0);
  g->ml_vertex.assign(nv, 0.0);
  for (int64_t e = 0; e < E; ++e) {
    double ne_d;
    if (n_elems) {
      if (n_elems[e] < 1) {
        delete g;
        return fail(GRF_EINVAL, "edge %lld has n_elems < 1", (long long)e);
      }
      ne_d = n_elems[e];
    } else {
      ne_d = std::ceil(lengths[e] / h);
      if (ne_d < 1) ne_d = 1;
      if (ne_d > 1e9) {
        delete g;
        return fail(GRF_EINVAL, "edge %lld needs too many elements", (long long)e);
      }
    }
    g->nel[e] = (int32_t)ne_d;
    g->he[e] = lengths[e] / ne_d;
    g->eu[e] = (int32_t)g->vertex_map[edge_u[e]];
    g->ev[e] = (int32_t)g->vertex_map[edge_v[e]];
    g->ioff[e + 1] = g->ioff[e] + (g->nel[e] - 1);
    g->ml_vertex[g->eu[e]] += 0.5 * g->he[e];
    g->ml_vertex[g->ev[e]] += 0.5 * g->he[e];
  }
  g->ni = g->ioff[E];
  // spectral bins: smallest bin whose limit holds the interior
  int32_t spec_mmax[kMaxBins];
  g->n_spec_bins = spec_bins(spec_mmax);
  {
    std::vector<std::vector<int32_t>> lists(g->n_spec_bins);
    for (int64_t e = 0; e < E; ++e) {
      const int64_t m = g->nel[e] - 1;
      for (int i = 0; i < g->n_spec_bins && m >= 1; ++i)
        if (m <= spec_mmax[i]) {
          lists[i].push_back((int32_t)e);
          break;
        }
    }
    for (int i = 0; i < g->n_spec_bins; ++i) {
      g->spec_count[i] = (int32_t)lists[i].size();
      g->spec_edges.insert(g->spec_edges.end(), lists[i].begin(), lists[i].end());
    }
  }
  const int64_t spec_limit = spec_mmax[g->n_spec_bins - 1];
  // recovery bins: smallest bin whose 32 * NW * B lanes x nodes hold the interior
  for (int p = 0; p < 3; ++p) {
    int32_t Bs[kMaxBins], NWs[kMaxBins];
    const int nb = recover_bins(p == 1, Bs, NWs);
    g->n_bins[p] = nb;
    std::vector<std::vector<int32_t>> lists(nb + 1);
    for (int64_t e = 0; e < E; ++e) {
      const int64_t m = g->nel[e] - 1;
      if (m <= 0) continue;
      if (p == 2 && m <= spec_limit) continue;  // left to the spectral path
      int bin = nb;
      for (int i = 0; i < nb; ++i)
        if (m <= (int64_t)32 * NWs[i] * Bs[i]) {
          bin = i;
          break;
        }
      lists[bin].push_back((int32_t)e);
    }
    for (int i = 0; i <= nb; ++i) {
      g->bin_count[p][i] = (int32_t)lists[i].size();
      g->bin_edges[p].insert(g->bin_edges[p].end(), lists[i].begin(), lists[i].end());
    }
  }
  g->n = nv + g->ni;
  // vertex incidence lists (CSR), edges in increasing id per vertex
  g->vptr.assign(nv + 1, 0);
  for (int64_t e = 0; e < E; ++e) {
    g->vptr[g->eu[e] + 1]++;
    g->vptr[g->ev[e] + 1]++;
  }
  for (int32_t v = 0; v < nv; ++v) g->vptr[v + 1] += g->vptr[v];
  g->adj_edge.resize(2 * E);
  g->adj_nbr.resize(2 * E);
  std::vector<int32_t> fill(g->vptr.begin(), g->vptr.end() - 1);
  for (int64_t e = 0; e < E; ++e) {
    const int32_t a = g->eu[e], b = g->ev[e];
    g->adj_edge[fill[a]] = (int32_t)e;
    g->adj_nbr[fill[a]++] = b;
    g->adj_edge[fill[b]] = (int32_t)e;
    g->adj_nbr[fill[b]++] = a;
  }
  // reverse incidence: the same edge seen from its other end
  g->adj_rev.assign(2 * E, -1);
  {
    std::vector<int32_t> first(E, -1);
    for (int32_t k = 0; k < 2 * (int32_t)E; ++k) {
      const int32_t e = g->adj_edge[k];
      if (first[e] < 0) {
        first[e] = k;
      } else {
        g->adj_rev[k] = first[e];
        g->adj_rev[first[e]] = k;
      }
    }
  }
  rcm_order(*g);
  *out = g;
  return GRF_OK;
}

int grf_graph_vertex_order(const grf_graph* g, int64_t* perm_out) {
  GRF_TRY(check_graph(g));
  if (!perm_out) return fail(GRF_EINVAL, "perm_out is null");
  for (int32_t i = 0; i < g->nv; ++i) perm_out[i] = g->rperm[i];
  return GRF_OK;
}

int grf_graph_destroy(grf_graph* g) {
  delete g;
  return GRF_OK;
}

int grf_graph_info(const grf_graph* g, int64_t* n_dofs, int64_t* n_kept_vertices,
                   int64_t* n_interior, int64_t* vertex_map, int64_t* interior_offsets) {
  GRF_TRY(check_graph(g));
  if (n_dofs) *n_dofs = g->n;
  if (n_kept_vertices) *n_kept_vertices = g->nv;
  if (n_interior) *n_interior = g->ni;
  if (vertex_map) std::memcpy(vertex_map, g->vertex_map.data(), sizeof(int64_t) * g->nv_in);
  if (interior_offsets)
    std::memcpy(interior_offsets, g->ioff.data(), sizeof(int64_t) * (g->ne + 1));
  return GRF_OK;
}

int grf_workspace_bytes(const grf_graph* g, double beta, double k_step, int64_t n_samples,
                        const grf_options* opts, size_t* bytes) {
  GRF_TRY(check_graph(g));
  if (!bytes) return fail(GRF_EINVAL, "bytes is null");
  Opts o;
  GRF_TRY(read_opts(opts, &o));
  GRF_TRY(check_params(1.0, beta, k_step));
  const size_t ts = o.precision == GRF_FP64 ? 8 : 4;
  std::vector<HostNodes> stages;
  plan(beta, k_step, &stages);
  size_t need = align_up((size_t)g->n * n_samples * ts);
  if (stages.size() > 1) need += align_up((size_t)g->n * n_samples * 8);
  size_t tail = 0;
  for (auto& s : stages) tail = std::max(tail, apply_bytes(g, s.L(), n_samples, ts, o));
  *bytes = need + tail;
  return GRF_OK;
}

int grf_sample(grf_graph* g, double kappa, double beta, double k_step, uint64_t seed,
               int64_t n_samples, void* out, const grf_options* opts, void* stream,
               grf_stats* stats) {
  GRF_TRY(check_graph(g));
  GRF_TRY(check_params(kappa, beta, k_step));
  Opts o;
  GRF_TRY(read_opts(opts, &o));
  if (n_samples < 0 || n_samples > (int64_t)1 << 24) return fail(GRF_EINVAL, "bad n_samples");
  if (n_samples == 0) return finish(RunStats{}, g, stats);
  if (!out) return fail(GRF_EINVAL, "out is null");
  GRF_TRY(ensure_device(g));
  cudaStream_t st = (cudaStream_t)stream;
  RunStats rs;
  rs.timing = o.timing;
  rs.mask = o.phase_mask;
  int r;
#define GRF_RUN(T, O)                                                                      \
  (o.use_graph ? sample_graph_impl<T, O>(g, kappa, beta, k_step, seed, n_samples, (O*)out, o, \
                                         st, &rs)                                          \
               : sample_impl<T, O>(g, kappa, beta, k_step, seed, n_samples, (O*)out, o, st, &rs))
  if (o.precision == GRF_FP64) {
    r = o.out_dtype == GRF_OUT_F64 ? GRF_RUN(double, double) : GRF_RUN(double, float);
  } else {
    r = o.out_dtype == GRF_OUT_F64 ? GRF_RUN(float, double) : GRF_RUN(float, float);
  }
#undef GRF_RUN
  if (r != GRF_OK) return r;
  return finish(rs, g, stats);
}

int grf_autotune(grf_graph* g, double kappa, double beta, double k_step, int64_t n_samples,
                 void* out, const grf_options* base, void* stream, int32_t reps,
                 grf_options* best, double* best_ms) {
  GRF_TRY(check_graph(g));
  GRF_TRY(check_params(kappa, beta, k_step));
  if (!best) return fail(GRF_EINVAL, "best is null");
  if (n_samples < 1 || !out) return fail(GRF_EINVAL, "need n_samples >= 1 and an out buffer");
  if (reps < 1) reps = 1;
  grf_options b0{};
  if (base) b0 = *base;
  b0.timing = 0;
  b0.use_graph = 0;
  Opts o;
  GRF_TRY(read_opts(&b0, &o));
  cudaStream_t st = (cudaStream_t)stream;
  const bool fp32 = o.precision == GRF_MIXED;
  std::vector<int> layouts = {GRF_PCG_PER_SYSTEM};
  if (fp32) {
    layouts.push_back(GRF_PCG_STAGED);
    layouts.push_back(GRF_PCG_STAGED_PAIRS);
    layouts.push_back(GRF_PCG_BATCHED);
  }
  // candidates (interior solver, recover_sg); recover_sg only matters for the
  // edges a solver leaves to the Thomas bins
  std::vector<std::pair<int, int>> cands;
  if (fp32) {
    for (int sg : {1, 2, 4}) cands.push_back({GRF_INTERIOR_THOMAS, sg});
    if (g->thomas_rest() > 0)
      for (int sg : {1, 2, 4}) cands.push_back({GRF_INTERIOR_SPECTRAL, sg});
    else
      cands.push_back({GRF_INTERIOR_SPECTRAL, 4});
    cands.push_back({GRF_INTERIOR_SPECTRAL_TC, 4});
    if (dst_gemm_sample_pad(n_samples) > 0) cands.push_back({GRF_INTERIOR_SPECTRAL_UMMA, 4});
  } else {
    cands.push_back({GRF_INTERIOR_THOMAS, 0});
  }
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  double best_t = 1e300;
  grf_options best_o = b0;
  int rc = GRF_OK;
  // three passes: the interior solvers with the default PCG layout, then the
  // PCG layouts with the best interior solver (the two phases hardly
  // interact), then, where FP32 tridiagonal edges remain, the layout of their
  // sweeps (segments only, node-parallel only, or the built-in length split)
  struct Trial {
    int lay, interior, sg, sweep;
  };
  std::vector<Trial> trials;
  for (auto cand : cands) trials.push_back({GRF_PCG_STAGED, cand.first, cand.second, b0.sweep});
  const size_t n_first = trials.size();
  size_t n_second = 0;
  for (size_t ti = 0;; ++ti) {
    if (ti == n_first) {
      for (int lay : layouts)
        if (lay != GRF_PCG_STAGED)
          trials.push_back({lay, best_o.interior, best_o.recover_sg, b0.sweep});
      n_second = trials.size();
    }
    if (n_second > 0 && ti == n_second && fp32) {
      const bool tridiag = best_o.interior == GRF_INTERIOR_THOMAS || g->thomas_rest() > 0;
      if (tridiag)
        for (int sw : {GRF_SWEEP_SEGMENTS, GRF_SWEEP_NODES})
          if (sw != b0.sweep)
            trials.push_back({best_o.pcg_layout, best_o.interior, best_o.recover_sg, sw});
    }
    if (ti >= trials.size()) break;
    {
      const Trial tr = trials[ti];
      grf_options c = b0;
      c.pcg_layout = tr.lay;
      c.interior = tr.interior;
      c.recover_sg = tr.sg;
      c.sweep = tr.sweep;
      rc = grf_sample(g, kappa, beta, k_step, 1, n_samples, out, &c, stream, nullptr);
      if (rc != GRF_OK && rc != GRF_ENOCONV) break;
      float ms = 0.f;
      if (cudaEventRecord(e0, st) != cudaSuccess) { rc = fail(GRF_ECUDA, "event record"); break; }
      for (int r = 0; r < reps && (rc == GRF_OK || rc == GRF_ENOCONV); ++r)
        rc = grf_sample(g, kappa, beta, k_step, 2 + r, n_samples, out, &c, stream, nullptr);
      if (rc != GRF_OK && rc != GRF_ENOCONV) break;
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      // the tensor-core condensation has to win by 3 %: on par, keep the
      // FP32 kernels (ties would otherwise flip from run to run)
      const double t = ms / reps * (c.interior == GRF_INTERIOR_SPECTRAL_TC ? 1.03 : 1.0);
      if (t < best_t) {
        best_t = t;
        best_o = c;
      }
    }
    if (rc != GRF_OK && rc != GRF_ENOCONV) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GRF_OK && rc != GRF_ENOCONV) return rc;
  if (base) {
    best_o.timing = base->timing;
    best_o.use_graph = base->use_graph;
  }
  *best = best_o;
  if (best_ms) *best_ms = best_t;
  return GRF_OK;
}

// The cached device output of the host entry points (grown when needed; a
// captured graph that writes the old buffer is dropped first).
static int ensure_host_out(grf_graph* g, size_t bytes, void* stream) {
  if (g->host_out_bytes >= bytes) return GRF_OK;
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  if (g->host_out) {
    CUDA_TRY(cudaDeviceSynchronize());
    g->drop_graph();
    CUDA_TRY(cudaFree(g->host_out));
    g->host_out = nullptr;
    g->host_out_bytes = 0;
  }
  CUDA_TRY(cudaMalloc(&g->host_out, bytes ? bytes : 1));
  g->host_out_bytes = bytes ? bytes : 1;
  return GRF_OK;
}

int grf_sample_host(grf_graph* g, double kappa, double beta, double k_step, uint64_t seed,
                    int64_t n_samples, void* out_host, const grf_options* opts, void* stream,
                    grf_stats* stats) {
  GRF_TRY(check_graph(g));
  if (!out_host) return fail(GRF_EINVAL, "out_host is null");
  Opts o;
  GRF_TRY(read_opts(opts, &o));
  GRF_TRY(ensure_device(g));
  const size_t bytes = (size_t)g->n * (size_t)n_samples * (o.out_dtype == GRF_OUT_F64 ? 8 : 4);
  GRF_TRY(ensure_host_out(g, bytes, stream));
  int r = grf_sample(g, kappa, beta, k_step, seed, n_samples, g->host_out, opts, stream, stats);
  if (r == GRF_OK || r == GRF_ENOCONV) {
    cudaError_t e = cudaMemcpyAsync(out_host, g->host_out, bytes, cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) r = fail(GRF_ECUDA, "copy to host: %s", cudaGetErrorString(e));
  }
  return r;
}

int grf_sample_host_stream(grf_graph* g, double kappa, double beta, double k_step,
                           const uint64_t* seeds, int64_t n_calls, int64_t n_samples,
                           void* const* out_host, const grf_options* opts, void* stream,
                           grf_stats* stats) {
  GRF_TRY(check_graph(g));
  if (n_calls < 0) return fail(GRF_EINVAL, "bad n_calls");
  if (n_calls == 0) return finish(RunStats{}, g, stats);
  if (!seeds || !out_host) return fail(GRF_EINVAL, "seeds or out_host is null");
  for (int64_t c = 0; c < n_calls; ++c)
    if (!out_host[c]) return fail(GRF_EINVAL, "out_host[%lld] is null", (long long)c);
  Opts o;
  GRF_TRY(read_opts(opts, &o));
  if (n_samples < 0 || n_samples > (int64_t)1 << 24) return fail(GRF_EINVAL, "bad n_samples");
  GRF_TRY(ensure_device(g));
  const size_t bytes = (size_t)g->n * (size_t)n_samples * (o.out_dtype == GRF_OUT_F64 ? 8 : 4);
  cudaStream_t st = (cudaStream_t)stream;
  GRF_TRY(ensure_host_out(g, bytes, stream));
  if (g->host_stage_bytes < bytes) {
    CUDA_TRY(cudaDeviceSynchronize());
    if (g->host_stage) CUDA_TRY(cudaFree(g->host_stage));
    g->host_stage = nullptr;
    g->host_stage_bytes = 0;
    CUDA_TRY(cudaMalloc(&g->host_stage, bytes ? bytes : 1));
    g->host_stage_bytes = bytes ? bytes : 1;
  }
  if (!g->copy_stream) {
    CUDA_TRY(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&g->ev_staged, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&g->ev_d2h, cudaEventDisableTiming));
  }
  grf_stats sum{};
  int worst = GRF_OK;
  for (int64_t c = 0; c < n_calls; ++c) {
    grf_stats one{};
    const int r = grf_sample(g, kappa, beta, k_step, seeds[c], n_samples, g->host_out, opts,
                             stream, &one);
    if (r != GRF_OK && r != GRF_ENOCONV) {
      cudaStreamSynchronize(g->copy_stream);
      return r;
    }
    if (r == GRF_ENOCONV) worst = r;
    sum.n_dofs = one.n_dofs;
    sum.n_nodes += one.n_nodes;
    sum.n_systems += one.n_systems;
    sum.pcg_iters_total += one.pcg_iters_total;
    sum.pcg_iters_max = std::max(sum.pcg_iters_max, one.pcg_iters_max);
    sum.n_unconverged += one.n_unconverged;
    sum.numeric_flag |= one.numeric_flag;
    sum.kernel_launches += one.kernel_launches;
    sum.n_precond_fallback += one.n_precond_fallback;
    for (int i = 0; i < 8; ++i) sum.phase_ms[i] += one.phase_ms[i];
    // stage the field (after the previous host copy has left the stage), then
    // copy it to the host on the copy stream while the next call computes
    if (c > 0) CUDA_TRY(cudaStreamWaitEvent(st, g->ev_d2h, 0));
    CUDA_TRY(cudaMemcpyAsync(g->host_stage, g->host_out, bytes, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaEventRecord(g->ev_staged, st));
    CUDA_TRY(cudaStreamWaitEvent(g->copy_stream, g->ev_staged, 0));
    CUDA_TRY(cudaMemcpyAsync(out_host[c], g->host_stage, bytes, cudaMemcpyDeviceToHost,
                             g->copy_stream));
    CUDA_TRY(cudaEventRecord(g->ev_d2h, g->copy_stream));
  }
  CUDA_TRY(cudaStreamSynchronize(g->copy_stream));
  if (stats) *stats = sum;
  return worst;
}

int grf_noise(grf_graph* g, uint64_t seed, int64_t n_samples, void* out, int32_t raw_words,
              void* stream) {
  GRF_TRY(check_graph(g));
  if (n_samples < 0) return fail(GRF_EINVAL, "bad n_samples");
  if (n_samples == 0) return GRF_OK;
  if (!out) return fail(GRF_EINVAL, "out is null");
  GRF_TRY(ensure_device(g));
  if (raw_words == 2) {  // consistent-mass noise W = R xi, FP32, written as double
    if (n_samples > 256) return fail(GRF_EINVAL, "at most 256 samples of consistent noise");
    GRF_TRY(ensure_cons_plan(g));
    const size_t need = align_up((size_t)g->n * n_samples * 4) +
                        align_up((size_t)g->nv * n_samples * 4);
    GRF_TRY(ensure_ws(g, need));
    Carve c(g->ws);
    float* b = c.take<float>((size_t)g->n * n_samples);
    float* wv = c.take<float>((size_t)g->nv * n_samples);
    cudaStream_t st = (cudaStream_t)stream;
    launch_noise_minor<float>(g->d, seed, n_samples, b, st, nullptr, g->cons.ones);
    launch_cons_noise(g->d, n_samples, b, wv, g->cons.rp, g->cons.rc, g->cons.rv, g->n_sm, st);
    launch_minor_to_major(g->n, n_samples, b, (double*)out, st);
    CUDA_TRY(cudaGetLastError());
    return GRF_OK;
  }
  if (raw_words != 0 && raw_words != 1) return fail(GRF_EINVAL, "raw_words must be 0, 1 or 2");
  launch_noise_major(g->d, seed, n_samples, out, raw_words != 0, (cudaStream_t)stream);
  CUDA_TRY(cudaGetLastError());
  return GRF_OK;
}

int grf_apply(grf_graph* g, double kappa, int64_t n_nodes, const double* alpha,
              const double* gamma, const double* weight, int64_t n_rhs, const double* rhs,
              void* out, const grf_options* opts, void* stream, grf_stats* stats) {
  GRF_TRY(check_graph(g));
  if (!(kappa > 0)) return fail(GRF_EINVAL, "kappa must be > 0");
  if (n_nodes < 1 || n_nodes > 100000 || !alpha || !gamma || !weight)
    return fail(GRF_EINVAL, "bad node list");
  for (int64_t l = 0; l < n_nodes; ++l)
    if (!(alpha[l] >= 0) || !(gamma[l] > 0) || !std::isfinite(alpha[l]) ||
        !std::isfinite(gamma[l]) || !std::isfinite(weight[l]))
      return fail(GRF_EINVAL, "node %lld needs alpha >= 0, gamma > 0", (long long)l);
  Opts o;
  GRF_TRY(read_opts(opts, &o));
  if (n_rhs < 0) return fail(GRF_EINVAL, "bad n_rhs");
  if (n_rhs == 0) return finish(RunStats{}, g, stats);
  if (!rhs || !out) return fail(GRF_EINVAL, "null buffer");
  GRF_TRY(ensure_device(g));
  HostNodes hn;
  hn.alpha.assign(alpha, alpha + n_nodes);
  hn.gamma.assign(gamma, gamma + n_nodes);
  hn.weight.assign(weight, weight + n_nodes);
  normalize_nodes(hn);
  GRF_TRY(check_fp32_range(g, o, kappa, std::vector<HostNodes>{hn}));
  const size_t ts = o.precision == GRF_FP64 ? 8 : 4;
  const size_t head = align_up((size_t)g->n * n_rhs * ts);
  if (o.consistent && (g->thomas_rest() > 0 || dst_gemm_sample_pad(n_rhs) == 0))
    return fail(GRF_ENOTSUP, "the consistent mass needs every edge within 1024 interior nodes "
                             "and at most 256 right-hand sides");
  GRF_TRY(ensure_ws(g, head + apply_bytes(g, hn.L(), n_rhs, ts, o)));
  if (o.spec_umma) GRF_TRY(ensure_dst_plan(g, n_rhs));
  cudaStream_t st = (cudaStream_t)stream;
  RunStats rs;
  rs.timing = o.timing;
  rs.mask = o.phase_mask;
  void* tail = (char*)g->ws + head;
  int r;
  if (o.precision == GRF_FP64) {
    double* b = (double*)g->ws;
    launch_to_minor<double>(g->d, n_rhs, rhs, b, false, st);
    r = o.out_dtype == GRF_OUT_F64 ? dd_apply<double, double>(g, hn, kappa, n_rhs, b, (double*)out, o, st, tail, &rs)
                                   : dd_apply<double, float>(g, hn, kappa, n_rhs, b, (float*)out, o, st, tail, &rs);
  } else {
    float* b = (float*)g->ws;
    launch_to_minor<float>(g->d, n_rhs, rhs, b, false, st);
    r = o.out_dtype == GRF_OUT_F64 ? dd_apply<float, double>(g, hn, kappa, n_rhs, b, (double*)out, o, st, tail, &rs)
                                   : dd_apply<float, float>(g, hn, kappa, n_rhs, b, (float*)out, o, st, tail, &rs);
  }
  if (r != GRF_OK) return r;
  return finish(rs, g, stats);
}

int grf_schur(grf_graph* g, double kappa, double alpha, double gamma, double* diag,
              double* offdiag, void* stream) {
  GRF_TRY(check_graph(g));
  if (!(kappa > 0) || !(alpha >= 0) || !(gamma > 0)) return fail(GRF_EINVAL, "bad parameters");
  if (!diag || !offdiag) return fail(GRF_EINVAL, "null buffer");
  GRF_TRY(ensure_device(g));
  HostNodes hn;
  hn.alpha = {alpha};
  hn.gamma = {gamma};
  hn.weight = {1.0};
  Opts o64{};
  o64.precision = GRF_FP64;
  GRF_TRY(ensure_ws(g, apply_bytes(g, 1, 1, 8, o64)));
  Carve c(g->ws);
  ApplyWs w;
  carve_apply(c, g, 1, 1, 8, &w);
  cudaStream_t st = (cudaStream_t)stream;
  GRF_TRY(upload_nodes(hn, w, st));
  launch_schur<double>(g->d, dev_nodes(w, 1), kappa * kappa, w.saa, offdiag, diag, w.offv,
                       nullptr, nullptr, nullptr, st);
  CUDA_TRY(cudaGetLastError());
  return GRF_OK;
}

int grf_vertex_solve(grf_graph* g, double kappa, double alpha, double gamma, int64_t n_rhs,
                     const double* rhs, double* g_out, double* u_out, const grf_options* opts,
                     void* stream, grf_stats* stats) {
  GRF_TRY(check_graph(g));
  if (!(kappa > 0) || !(alpha >= 0) || !(gamma > 0)) return fail(GRF_EINVAL, "bad parameters");
  Opts o;
  GRF_TRY(read_opts(opts, &o));
  if (n_rhs < 0) return fail(GRF_EINVAL, "bad n_rhs");
  if (n_rhs == 0) return finish(RunStats{}, g, stats);
  if (!rhs || !g_out || !u_out) return fail(GRF_EINVAL, "null buffer");
  GRF_TRY(ensure_device(g));
  HostNodes hn;
  hn.alpha = {alpha};
  hn.gamma = {gamma};
  hn.weight = {1.0};
  const size_t ts = o.precision == GRF_FP64 ? 8 : 4;
  const size_t head = align_up((size_t)g->n * n_rhs * ts);
  GRF_TRY(ensure_ws(g, head + apply_bytes(g, 1, n_rhs, ts, o)));
  Carve c((char*)g->ws + head);
  ApplyWs w;
  carve_apply(c, g, 1, n_rhs, ts, &w, o.precond, o.spectral);
  cudaStream_t st = (cudaStream_t)stream;
  GRF_TRY(upload_nodes(hn, w, st));
  const double k2 = kappa * kappa;
  RunStats rs;
  rs.timing = o.timing;
  rs.mask = o.phase_mask;
  rs.launches += 1;
  if (o.precision == GRF_FP64) {
    double* b = (double*)g->ws;
    launch_to_minor<double>(g->d, n_rhs, rhs, b, false, st);
    GRF_TRY(vertex_phase<double>(g, w, 1, k2, n_rhs, b, g_out, u_out, o, st, &rs));
  } else {
    float* b = (float*)g->ws;
    launch_to_minor<float>(g->d, n_rhs, rhs, b, false, st);
    GRF_TRY(vertex_phase<float>(g, w, 1, k2, n_rhs, b, g_out, u_out, o, st, &rs));
  }
  GRF_TRY(collect(w, st, 1, n_rhs, &rs));
  return finish(rs, g, stats);
}

// grf_vertex_solve without any device allocation: every scratch buffer lives
// in grf_noalloc_scratch. The graph must already be resident on the current
// device. The first call on a device looks up the array's device address
// (cudaGetSymbolAddress); make that first call before any stream capture.
// Calls share the array, so calls that overlap on the GPU race with each
// other; the PCG status words are cleared at every call, everything else is
// fully overwritten before it is read. Per-phase timing is not recorded here.
int grf_vertex_solve_noalloc(grf_graph* g, double kappa, double alpha, double gamma,
                             int64_t n_rhs, const double* rhs, double* g_out, double* u_out,
                             const grf_options* opts, void* stream, grf_stats* stats) {
  GRF_TRY(check_graph(g));
  if (!(kappa > 0) || !(alpha >= 0) || !(gamma > 0)) return fail(GRF_EINVAL, "bad parameters");
  Opts o;
  GRF_TRY(read_opts(opts, &o));
  if (n_rhs < 0) return fail(GRF_EINVAL, "bad n_rhs");
  if (n_rhs == 0) return finish(RunStats{}, g, stats);
  if (!rhs || !g_out || !u_out) return fail(GRF_EINVAL, "null buffer");
  if (o.precond != GRF_PRECOND_JACOBI)
    return fail(GRF_ENOTSUP, "grf_vertex_solve_noalloc supports GRF_PRECOND_JACOBI only");
  const size_t ts = o.precision == GRF_FP64 ? 8 : 4;
  Carve dry(nullptr);
  ApplyWs w;
  void* bptr = nullptr;
  carve_vertex_solve(dry, g, n_rhs, ts, &w, &bptr);
  if (dry.off > kNoAllocScratchBytes)
    return fail(GRF_EINVAL,
                "grf_vertex_solve_noalloc needs %zu bytes of scratch for n_dofs=%lld x n_rhs=%lld "
                "but its static scratch holds %zu bytes; use grf_vertex_solve or fewer rhs",
                dry.off, (long long)g->n, (long long)n_rhs, kNoAllocScratchBytes);
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (g->device != dev || !g->dev_block)
    return fail(GRF_EINVAL,
                "graph is not resident on device %d; a call that allocates (e.g. grf_vertex_solve) "
                "must have used it there first", dev);
  void* base = nullptr;
  GRF_TRY(noalloc_scratch(dev, &base));
  Carve c(base);
  carve_vertex_solve(c, g, n_rhs, ts, &w, &bptr);
  cudaStream_t st = (cudaStream_t)stream;
  const double one = 1.0;
  CUDA_TRY(cudaMemcpyAsync(w.alpha, &alpha, sizeof(double), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(w.gamma, &gamma, sizeof(double), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(w.weight, &one, sizeof(double), cudaMemcpyHostToDevice, st));
  const double k2 = kappa * kappa;
  RunStats rs;
  rs.timing = false;
  rs.launches += 1;
  if (o.precision == GRF_FP64) {
    double* b = (double*)bptr;
    launch_to_minor<double>(g->d, n_rhs, rhs, b, false, st);
    GRF_TRY(vertex_phase<double>(g, w, 1, k2, n_rhs, b, g_out, u_out, o, st, &rs));
  } else {
    float* b = (float*)bptr;
    launch_to_minor<float>(g->d, n_rhs, rhs, b, false, st);
    GRF_TRY(vertex_phase<float>(g, w, 1, k2, n_rhs, b, g_out, u_out, o, st, &rs));
  }
  GRF_TRY(collect(w, st, 1, n_rhs, &rs));
  return finish(rs, g, stats);
}

}  // extern "C"
