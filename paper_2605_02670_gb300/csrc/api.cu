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

}  // namespace

struct grf_graph {
  int64_t nv_in = 0;
  int32_t nv = 0;
  int32_t ne = 0;
  int64_t ni = 0;
  int64_t n = 0;
  std::vector<int64_t> vertex_map;
  std::vector<int32_t> eu, ev, nel, vptr, adj_edge, adj_nbr;
  std::vector<double> he;
  std::vector<int64_t> ioff;
  std::vector<double> ml_vertex;  // lumped mass at kept vertices
  // recovery edge bins per precision ([0] FP32 sweeps, [1] FP64): edge ids
  // grouped by bin, the count per bin, and last the edges beyond every bin
  std::vector<int32_t> bin_edges[2];
  int32_t bin_count[2][kMaxBins + 1] = {};
  int32_t n_bins[2] = {0, 0};
  const int32_t* d_bin_edges[2] = {nullptr, nullptr};

  int64_t long_edges(bool fp64) const { return bin_count[fp64 ? 1 : 0][n_bins[fp64 ? 1 : 0]]; }

  int device = -1;
  void* dev_block = nullptr;
  DevGraph d{};
  void* ws = nullptr;
  size_t ws_bytes = 0;

  // Captured launch sequence of one grf_sample configuration (options.use_graph).
  // Device pointers (workspace, output, node arrays) are baked into the graph,
  // so any change of them or of the configuration re-captures.
  struct GraphCache {
    bool valid = false;
    int precision = 0, out_dtype = 0, pcg_layout = 0, recover_sg = 0, max_iter = 0;
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
  } gc;
  cudaStream_t cap_stream = nullptr;

  void drop_graph() {
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    if (gc.nodes_dev) cudaFree(gc.nodes_dev);
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
      cudaSetDevice(cur);
    }
  }
};

namespace {

__global__ void sqrt_ml_kernel(DevGraph g, const double* mlv, double* out) {
  const int64_t total = g.n;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total;
       j += (int64_t)gridDim.x * blockDim.x) {
    if (j < g.nv) {
      out[j] = sqrt(mlv[j]);
    } else {
      // interior DOF: find its edge by bisection over the interior offsets
      const int64_t i = j - g.nv;
      int32_t lo = 0, hi = g.ne - 1;
      while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (g.ioff[mid] <= i) lo = mid; else hi = mid - 1;
      }
      out[j] = sqrt(g.he[lo]);
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
  c.take<int32_t>(E + 1); c.take<int32_t>(E + 1);
  void* blk = nullptr;
  CUDA_TRY(cudaMalloc(&blk, c.off));
  g->device = dev;
  g->dev_block = blk;
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
  for (int p = 0; p < 2; ++p) {
    int32_t* be = k.take<int32_t>(E + 1);
    if (!g->bin_edges[p].empty())
      CUDA_TRY(cudaMemcpy(be, g->bin_edges[p].data(), g->bin_edges[p].size() * 4,
                          cudaMemcpyHostToDevice));
    g->d_bin_edges[p] = be;
  }
  CUDA_TRY(cudaMemcpy(eu, g->eu.data(), E * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(ev, g->ev.data(), E * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(nel, g->nel.data(), E * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(he, g->he.data(), E * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(ioff, g->ioff.data(), (E + 1) * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(vptr, g->vptr.data(), (V + 1) * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(ae, g->adj_edge.data(), 2 * E * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(an, g->adj_nbr.data(), 2 * E * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(mlv, g->ml_vertex.data(), V * 8, cudaMemcpyHostToDevice));
  DevGraph& d = g->d;
  d.nv = g->nv; d.ne = g->ne; d.ni = g->ni; d.n = g->n;
  d.max_m = 0;
  for (int32_t e = 0; e < g->ne; ++e) d.max_m = std::max(d.max_m, g->nel[e] - 1);
  d.eu = eu; d.ev = ev; d.nel = nel; d.he = he; d.ioff = ioff;
  d.vptr = vptr; d.adj_edge = ae; d.adj_nbr = an; d.sqrt_ml = sml;
  int64_t blocks = (g->n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  sqrt_ml_kernel<<<(int)blocks, 256>>>(d, mlv, sml);
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

struct HostNodes {
  std::vector<double> alpha, gamma, weight;
  int32_t L() const { return (int32_t)alpha.size(); }
};

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
  int pcg_layout;  // 1 per system, 2 staged
  int recover_sg;  // 1, 2 or 4
  bool use_graph;
};

int read_opts(const grf_options* o, Opts* r) {
  r->use_graph = o && o->use_graph != 0;
  r->timing = o && o->timing != 0 && !r->use_graph;
  const int sg = o ? o->recover_sg : 0;
  if (sg != 0 && sg != 1 && sg != 2 && sg != 4)
    return fail(GRF_EINVAL, "recover_sg must be 0, 1, 2 or 4 (got %d)", sg);
  r->recover_sg = sg == 0 ? 4 : sg;
  const int lay = o ? o->pcg_layout : GRF_PCG_AUTO;
  if (lay < GRF_PCG_AUTO || lay > GRF_PCG_STAGED)
    return fail(GRF_EINVAL, "unknown pcg_layout %d", lay);
  r->pcg_layout = lay == GRF_PCG_AUTO ? GRF_PCG_PER_SYSTEM : lay;
  r->precision = o ? o->precision : GRF_FP64;
  r->precond = o ? o->precond : GRF_PRECOND_JACOBI;
  r->out_dtype = o ? o->out_dtype : GRF_OUT_F64;
  r->max_iter = (o && o->max_iter > 0) ? o->max_iter : 1000;
  r->rtol = (o && o->rtol > 0) ? o->rtol : (r->precision == GRF_FP64 ? 1e-12 : 1e-9);
  if (r->precision != GRF_FP64 && r->precision != GRF_MIXED)
    return fail(GRF_EINVAL, "unknown precision %d", r->precision);
  if (r->precond != GRF_PRECOND_JACOBI)
    return fail(GRF_ENOTSUP, "preconditioner %d not available", r->precond);
  if (r->out_dtype != GRF_OUT_F64 && r->out_dtype != GRF_OUT_F32)
    return fail(GRF_EINVAL, "unknown out_dtype %d", r->out_dtype);
  return GRF_OK;
}

// Device workspace of one domain-decomposed apply with L nodes and S right-hand sides.
struct ApplyWs {
  double *alpha, *gamma, *weight, *saa, *sab, *diag, *offv, *gvec, *x, *acc;
  void *r, *p, *q, *d;  // PCG vectors in the sweep precision T [L][S][V]
  void* dscale;         // T [L][V]
  void* offv_t;         // float [L][2E] (mixed precision only)
  void *yscr, *rpscr;
  void* prm;  // SweepParams<T> [L][E]
  void* xw;   // T [L][S][V]
  int32_t* iters;
  PcgStatus* status;
};

void carve_apply(Carve& c, const grf_graph* g, int32_t L, int64_t S, size_t tsize, ApplyWs* w) {
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
  w->r = c.take<char>(Ls * Ss * V * tsize);
  w->p = c.take<char>(Ls * Ss * V * tsize);
  w->q = c.take<char>(Ls * Ss * V * tsize);
  w->d = c.take<char>(Ls * Ss * V * tsize);
  w->dscale = c.take<char>(Ls * V * tsize);
  w->offv_t = tsize == 4 ? c.take<char>(Ls * 2 * E * 4) : nullptr;
  // scratch of the sequential recovery, only for edges longer than every bin
  const size_t ni_long = g->long_edges(tsize == 8) > 0 ? (size_t)g->ni : 0;
  w->acc = c.take<double>(ni_long * Ss);
  w->yscr = c.take<char>(ni_long * Ss * tsize);
  w->rpscr = c.take<char>(ni_long * nsg * tsize);
  w->prm = c.take<char>(Ls * E * 4 * tsize);
  w->xw = c.take<char>(Ls * Ss * V * tsize);
  w->iters = c.take<int32_t>(Ls * Ss);
  w->status = c.take<PcgStatus>(1);
}

// Per-call statistics, kernel-launch count and (optional) CUDA-event phase timing.
struct RunStats {
  int64_t nodes = 0, systems = 0, iters_total = 0;
  int32_t iters_max = 0, unconverged = 0, numeric = 0, launches = 0;
  bool timing = false;
  // graph capture: status words are copied to pinned host slots, no syncs
  bool capturing = false;
  PcgStatus* h_status = nullptr;
  int stage_idx = 0;
  struct Span {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Span> spans;
  cudaEvent_t open = nullptr;
  double phase_ms[6] = {0, 0, 0, 0, 0, 0};

  void begin(cudaStream_t st) {
    if (!timing) return;
    cudaEventCreate(&open);
    cudaEventRecord(open, st);
  }
  void end(int phase, cudaStream_t st) {
    if (!timing || !open) return;
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, st);
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
  rs->iters_total += (int64_t)h.iters_total;
  if (h.iters_max > rs->iters_max) rs->iters_max = h.iters_max;
  rs->unconverged += h.n_unconverged;
  rs->numeric += h.numeric_flag;
  return GRF_OK;
}

// Schur blocks + condensation + PCG for the nodes already uploaded to w.
template <typename T>
int vertex_phase(grf_graph* g, const ApplyWs& w, int32_t L, double kappa2, int64_t S,
                 const T* b, double* gvec, double* xv, const Opts& o, cudaStream_t st,
                 RunStats* rs) {
  const DevNodes nd = dev_nodes(w, L);
  rs->begin(st);
  rs->launches += launch_schur<T>(g->d, nd, kappa2, w.saa, w.sab, w.diag, w.offv,
                                  (SweepParams<T>*)w.prm, (T*)w.dscale, (T*)w.offv_t, st);
  rs->end(1, st);
  rs->begin(st);
  launch_condense<T>(g->d, nd, kappa2, S, b, gvec, st);
  rs->end(2, st);
  CUDA_TRY(cudaMemsetAsync(w.status, 0, sizeof(PcgStatus), st));
  // FP64 PCG uses the FP64 blocks; the FP32 solve their scaled FP32 copy
  const T* offv_t = sizeof(T) == 8 ? (const T*)w.offv : (const T*)w.offv_t;
  rs->begin(st);
  launch_pcg<T>(g->d, L, S, w.diag, w.offv, (const T*)w.dscale, offv_t, gvec, xv, (T*)w.d,
                (T*)w.r, (T*)w.p, (T*)w.q, o.rtol, o.max_iter, w.iters, w.status,
                o.pcg_layout, st);
  rs->end(3, st);
  rs->launches += 3;
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
  carve_apply(c, g, hn.L(), S, sizeof(T), &w);
  const double k2 = kappa * kappa;
  if (nodes_dev) {
    w.alpha = const_cast<double*>(nodes_dev);
    w.gamma = const_cast<double*>(nodes_dev) + hn.L();
    w.weight = const_cast<double*>(nodes_dev) + 2 * hn.L();
  } else {
    GRF_TRY(upload_nodes(hn, w, st));
  }
  GRF_TRY(vertex_phase<T>(g, w, hn.L(), k2, S, b, w.gvec, w.x, o, st, rs));
  const int p = sizeof(T) == 8 ? 1 : 0;
  rs->begin(st);
  rs->launches += launch_recover<T, OutT>(g->d, dev_nodes(w, hn.L()), k2, S, b, w.x, out,
                                          (const SweepParams<T>*)w.prm, (T*)w.xw,
                                          g->d_bin_edges[p], g->bin_count[p], g->n_bins[p], w.acc,
                                          (T*)w.yscr, (T*)w.rpscr, o.recover_sg, st);
  rs->end(4, st);
  CUDA_TRY(cudaGetLastError());
  return collect(w, st, hn.L(), S, rs);
}

size_t apply_bytes(const grf_graph* g, int32_t L, int64_t S, size_t tsize) {
  Carve c(nullptr);
  ApplyWs w;
  carve_apply(c, g, L, S, tsize, &w);
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
    for (int i = 0; i < 6; ++i) stats->phase_ms[i] = rs.phase_ms[i];
  }
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
                       size_t tsize) {
  size_t need = align_up((size_t)g->n * S * tsize);
  size_t tail = 0;
  for (auto& s : stages) tail = std::max(tail, apply_bytes(g, s.L(), S, tsize));
  if (stages.size() > 1) need += align_up((size_t)g->n * S * sizeof(double));
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
  void* ws_tail = g->ws ? (char*)g->ws + c.off : nullptr;
  rs->begin(st);
  launch_noise_minor<T>(g->d, seed, S, b, st, seed_dev);
  rs->end(0, st);
  rs->launches += 1;
  CUDA_TRY(cudaGetLastError());
  for (size_t i = 0; i < stages.size(); ++i) {
    const bool last = i + 1 == stages.size();
    const double* nd = nodes_dev ? (*nodes_dev)[i] : nullptr;
    if (i > 0) {
      rs->begin(st);
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
  GRF_TRY(ensure_ws(g, sample_ws_bytes(g, stages, S, sizeof(T))));
  return enqueue_sample<T, OutT>(g, stages, kappa, seed, S, out, o, st, rs);
}

// The same call through a captured CUDA graph: captured once per configuration
// (on an internal stream), then replayed on the caller's stream with the seed
// copied in from pinned memory. Iteration statistics come back through pinned
// status slots; per-phase timing is not available on this path.
template <typename T, typename OutT>
int sample_graph_impl(grf_graph* g, double kappa, double beta, double k_step, uint64_t seed,
                      int64_t S, OutT* out, const Opts& o, cudaStream_t st, RunStats* rs) {
  std::vector<HostNodes> stages;
  plan(beta, k_step, &stages);
  GRF_TRY(ensure_ws(g, sample_ws_bytes(g, stages, S, sizeof(T))));
  auto& gc = g->gc;
  const bool hit = gc.valid && gc.precision == o.precision && gc.out_dtype == o.out_dtype &&
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
    RunStats cap;
    cap.capturing = true;
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
    gc.stage_L.clear();
    for (auto& s : stages) gc.stage_L.push_back(s.L());
    gc.launches = cap.launches;
    gc.precision = o.precision;
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
  w->r = c.take<char>(Ss * V * tsize);
  w->p = c.take<char>(Ss * V * tsize);
  w->q = c.take<char>(Ss * V * tsize);
  w->d = c.take<char>(Ss * V * tsize);
  w->dscale = c.take<char>(V * tsize);
  w->offv_t = tsize == 4 ? c.take<char>(2 * E * 4) : nullptr;
  w->iters = c.take<int32_t>(Ss);
  w->status = c.take<PcgStatus>(1);
  w->gvec = w->x = w->acc = nullptr;
  w->yscr = w->rpscr = nullptr;
  w->prm = w->xw = nullptr;
}

}  // namespace

extern "C" {

const char* grf_last_error(void) { return g_last_error.c_str(); }

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
  // recovery bins: smallest bin whose 32 * NW * B lanes x nodes hold the interior
  for (int p = 0; p < 2; ++p) {
    int32_t Bs[kMaxBins], NWs[kMaxBins];
    const int nb = recover_bins(p == 1, Bs, NWs);
    g->n_bins[p] = nb;
    std::vector<std::vector<int32_t>> lists(nb + 1);
    for (int64_t e = 0; e < E; ++e) {
      const int64_t m = g->nel[e] - 1;
      if (m <= 0) continue;
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
  *out = g;
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
  for (auto& s : stages) tail = std::max(tail, apply_bytes(g, s.L(), n_samples, ts));
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
  if (fp32) layouts.push_back(GRF_PCG_STAGED);
  std::vector<int> sgs = fp32 ? std::vector<int>{1, 2, 4} : std::vector<int>{2};
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  double best_t = 1e300;
  grf_options best_o = b0;
  int rc = GRF_OK;
  for (int lay : layouts) {
    for (int sg : sgs) {
      grf_options c = b0;
      c.pcg_layout = lay;
      c.recover_sg = fp32 ? sg : 0;
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
      const double t = ms / reps;
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

int grf_sample_host(grf_graph* g, double kappa, double beta, double k_step, uint64_t seed,
                    int64_t n_samples, void* out_host, const grf_options* opts, void* stream,
                    grf_stats* stats) {
  GRF_TRY(check_graph(g));
  if (!out_host) return fail(GRF_EINVAL, "out_host is null");
  Opts o;
  GRF_TRY(read_opts(opts, &o));
  GRF_TRY(ensure_device(g));
  const size_t bytes = (size_t)g->n * (size_t)n_samples * (o.out_dtype == GRF_OUT_F64 ? 8 : 4);
  void* dout = nullptr;
  CUDA_TRY(cudaMallocAsync(&dout, bytes ? bytes : 1, (cudaStream_t)stream));
  int r = grf_sample(g, kappa, beta, k_step, seed, n_samples, dout, opts, stream, stats);
  if (r == GRF_OK || r == GRF_ENOCONV) {
    cudaError_t e = cudaMemcpyAsync(out_host, dout, bytes, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) r = fail(GRF_ECUDA, "copy to host: %s", cudaGetErrorString(e));
  }
  cudaFreeAsync(dout, (cudaStream_t)stream);
  return r;
}

int grf_noise(grf_graph* g, uint64_t seed, int64_t n_samples, void* out, int32_t raw_words,
              void* stream) {
  GRF_TRY(check_graph(g));
  if (n_samples < 0) return fail(GRF_EINVAL, "bad n_samples");
  if (n_samples == 0) return GRF_OK;
  if (!out) return fail(GRF_EINVAL, "out is null");
  GRF_TRY(ensure_device(g));
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
  const size_t ts = o.precision == GRF_FP64 ? 8 : 4;
  const size_t head = align_up((size_t)g->n * n_rhs * ts);
  GRF_TRY(ensure_ws(g, head + apply_bytes(g, hn.L(), n_rhs, ts)));
  cudaStream_t st = (cudaStream_t)stream;
  RunStats rs;
  rs.timing = o.timing;
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
  GRF_TRY(ensure_ws(g, apply_bytes(g, 1, 1, 8)));
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
  GRF_TRY(ensure_ws(g, head + apply_bytes(g, 1, n_rhs, ts)));
  Carve c((char*)g->ws + head);
  ApplyWs w;
  carve_apply(c, g, 1, n_rhs, ts, &w);
  cudaStream_t st = (cudaStream_t)stream;
  GRF_TRY(upload_nodes(hn, w, st));
  const double k2 = kappa * kappa;
  RunStats rs;
  rs.timing = o.timing;
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
