/*
 * grf.h -- C ABI of the GB300 (sm_103a) sampler of Matern-type Gaussian random
 * fields on metric graphs: lumped-mass FEM white noise, sinc quadrature of the
 * Balakrishnan integral, and a non-overlapping edge/vertex domain decomposition
 * of every shifted system (Kovacs, Molnar, Szaraz, "Efficient generation of
 * Gaussian random fields on metric graphs via domain decomposition and mass
 * matrix lumping").
 *
 * Conventions used below.
 *   M_L  lumped mass: h_e at an interior node of edge e, sum_{e at v} h_e/2 at
 *        vertex v (Sec. 3, Phase 2, lumped case).
 *   G    P1 stiffness (Sec. 3, Phase 2);  K = kappa^2 M_L + G (the operator
 *        kappa^2 - Delta of Eq. 1).
 *   b    white noise M_L^{1/2} xi, xi ~ N(0, I) (Eq. wh_def, Sec. 2.5).
 *   Quadrature (Eq. 4 and the limits of Sec. 4.1), 0 < beta < 1:
 *        y_l = l k, l = -K^-..K^+, K^- = ceil(pi^2/(4k^2 beta)),
 *        K^+ = ceil(pi^2/(4k^2(1-beta))), t_l = e^{2 y_l},
 *        w_l = (2k sin(pi beta)/pi) e^{2 beta y_l};
 *        U = sum_l w_l (M_L + t_l K)^{-1} b   (= sum_l (c_I M_L + c_L K)^{-1} b).
 *   beta >= 1: beta = n + f; U = (K^{-1} M_L)^n U_f (f > 0) or
 *        (K^{-1} M_L)^{n-1} K^{-1} b (f = 0).
 *   DOF order: kept vertices (degree-0 vertices are dropped) in increasing
 *        input id, then the interior nodes edge by edge, each edge from
 *        edge_u towards edge_v (Sec. 3, Phase 1 mesh).
 *   Field buffers are sample-major: element (s, j) at s * n_dofs + j.
 *
 * Ownership: input host arrays are copied; a grf_graph is owned by the library
 * until grf_graph_destroy; output buffers and streams belong to the caller.
 * The library allocates and caches device memory per graph (graph arrays and
 * workspace), freed by grf_graph_destroy.
 *
 * Errors: every entry point returns GRF_OK (0) or a negative code; the
 * message of the last failure on the calling thread is in grf_last_error().
 * Device pointers must be on the device that is current when the call is made.
 * All device work is enqueued on `stream` (NULL = legacy default stream);
 * calls that return statistics synchronise that stream before returning.
 */
#ifndef GRF_H
#define GRF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRF_OK 0
#define GRF_EINVAL (-1)   /* invalid argument */
#define GRF_ENOMEM (-2)   /* device or host allocation failed */
#define GRF_ENOCONV (-3)  /* some vertex PCG did not reach rtol in max_iter; output written */
#define GRF_ECUDA (-4)    /* CUDA runtime error */
#define GRF_ENOTSUP (-5)  /* option not supported */
#define GRF_ENUMERIC (-6) /* NaN/Inf or loss of positive definiteness detected */

#define GRF_FP64 0        /* every step in FP64 */
#define GRF_MIXED 1       /* FP32 edge sweeps; FP64 Schur blocks, PCG, quadrature sum */

#define GRF_PRECOND_JACOBI 0   /* z = D^-1 r */
#define GRF_PRECOND_LEARNED 1  /* z = B B^T r on the Jacobi-scaled system, B from the network
                                  of grf_precond_* (GRF_MIXED only; see below) */
#define GRF_PRECOND_NEUMANN 2  /* the paper's Neumann-Neumann preconditioner (Sec. 3, Phase 4,
                                  Neumann step): z = D_G^-1 (sum_e (S^(e))^-1) D_G^-1 r with
                                  D_G = diag(vertex degree) and the exact 2x2 edge blocks
                                  S^(e); on the Jacobi-scaled system in GRF_MIXED */

#define GRF_OUT_F64 0
#define GRF_OUT_F32 1

typedef struct grf_graph grf_graph;

typedef struct grf_options {
  int32_t precision;   /* GRF_FP64 or GRF_MIXED */
  int32_t precond;     /* GRF_PRECOND_JACOBI, GRF_PRECOND_LEARNED or GRF_PRECOND_NEUMANN */
  int32_t out_dtype;   /* GRF_OUT_F64 or GRF_OUT_F32 */
  int32_t max_iter;    /* PCG iteration cap per system; <= 0: 1000 */
  double rtol;         /* PCG stop: ||r||_2 <= rtol ||g||_2; <= 0: 1e-12 (FP64) / 1e-8 (mixed) */
  int32_t timing;      /* nonzero: record CUDA events around each phase (grf_stats.phase_ms);
                          GRF_TIMING_ONLY | mask: only around the phases whose bit p
                          (p = the phase_ms index, bits 0-7) is set; other bits: GRF_EINVAL */
  int32_t pcg_layout;  /* GRF_PCG_AUTO, _PER_SYSTEM, _STAGED, _STAGED_PAIRS, _BATCHED (below) */
  int32_t recover_sg;  /* samples per lane in the interior recovery: 0 = auto, or 1, 2, 4
                          (FP32 sweeps; FP64 sweeps always use 2) */
  int32_t use_graph;   /* grf_sample only: nonzero captures the call's launch sequence into a
                          CUDA graph cached on the handle (re-captured when the parameters,
                          options, sample count or output pointer change) and replays it;
                          with timing, the phase events are event record nodes of the
                          graph and every replay reports its own phase_ms */
  int32_t interior;    /* edge-interior solver of the condensation and recovery steps:
                          GRF_INTERIOR_AUTO, GRF_INTERIOR_THOMAS, GRF_INTERIOR_SPECTRAL,
                          GRF_INTERIOR_SPECTRAL_TC or GRF_INTERIOR_SPECTRAL_UMMA */
  int32_t sweep;       /* how FP32 edges left to the tridiagonal solves are swept:
                          GRF_SWEEP_AUTO, GRF_SWEEP_SEGMENTS or GRF_SWEEP_NODES */
  int32_t mass;        /* GRF_MASS_LUMPED (the method) or GRF_MASS_CONSISTENT (the paper's
                          comparison system, below) */
} grf_options;

/* Mass matrix of the noise and the operator:
 *   LUMPED: M_L (Sec. 2.5 mass lumping), noise b = M_L^{1/2} xi;
 *   CONSISTENT: the consistent mass of Sec. 3 Phase 2 in the noise, W = R xi
 *     with M = R R^T the Cholesky factor in the order interiors (edge by edge),
 *     then vertices by kept id, and in the operator, A_l = M + t_l (kappa^2 M + G).
 *     Runs with GRF_MIXED, GRF_PRECOND_JACOBI, interior AUTO or SPECTRAL_UMMA,
 *     0 < beta < 1, at most 256 samples per call and every edge within 1024
 *     interior nodes (else GRF_ENOTSUP). Its first use on a graph factors the
 *     vertex Schur complement of the mass on the host (envelope Cholesky in
 *     kept-vertex order; GRF_ENOTSUP above 2^27 envelope entries). */
#define GRF_MASS_LUMPED 0
#define GRF_MASS_CONSISTENT 1

/* Edge-interior solvers (same results up to rounding):
 *   THOMAS: per node l a tridiagonal elimination along the edge (Sec. 3, Phases
 *     3 and 5 as printed);
 *   SPECTRAL (GRF_MIXED only): the interior blocks of all nodes share the
 *     discrete sine transform's eigenvectors on a uniform edge mesh, so the
 *     sum over nodes is applied as one sine-transform pair per edge and sample
 *     plus a dense (interior nodes x nodes) by (nodes x samples) contraction;
 *     edges with more than 1024 interior nodes still use THOMAS;
 *   AUTO: SPECTRAL in GRF_MIXED, THOMAS in GRF_FP64. */
#define GRF_INTERIOR_AUTO 0
#define GRF_INTERIOR_THOMAS 1
#define GRF_INTERIOR_SPECTRAL 2
#define GRF_INTERIOR_SPECTRAL_TC 3  /* SPECTRAL with the condensation's sine transform
                                       and end-value contraction on the tensor cores
                                       (mma.sync, TF32 operands in three terms); the
                                       recovery as SPECTRAL */
#define GRF_INTERIOR_SPECTRAL_UMMA 4 /* SPECTRAL with both sine transforms of every edge
                                        as tcgen05 tensor-core products: the edges are
                                        grouped by interior-node count m and each group's
                                        transforms are one product with Phi_m (BF16 hi/lo
                                        operands in three terms, FP32 accumulation in
                                        tensor memory); the end values and the sine-basis
                                        coefficients as SPECTRAL. Needs n_samples <= 256
                                        (larger sample counts run as SPECTRAL) */

/* Parallel layouts of the FP32 tridiagonal edge solves (same results up to
 * rounding; FP64 sweeps always use SEGMENTS):
 *   SEGMENTS: the lanes of up to 16 warps split one edge into segments, the
 *     eliminations of one node at a time run as scans across the lanes, and
 *     the sum over nodes stays in registers;
 *   NODES: one warp per edge and group of 4 samples, each lane a set of nodes
 *     (at most 256 nodes) swept along the whole edge; the recovery uses the
 *     twisted factorisation x_K = (y_K + z_K - r_K) / gamma_K (one elimination
 *     from each end, no back substitution) and sums over nodes across lanes;
 *   AUTO: NODES for edges with more than 64 interior nodes, SEGMENTS below. */
#define GRF_SWEEP_AUTO 0
#define GRF_SWEEP_SEGMENTS 1
#define GRF_SWEEP_NODES 2

/* Vertex PCG launch layouts (same results up to rounding):
 *   PER_SYSTEM: one CTA per (node, sample) system, Schur matrix read through
 *     the caches, vectors in shared memory when they fit;
 *   STAGED (mixed precision, Jacobi, graphs up to 4096 kept vertices whose
 *     Schur matrix fits in shared memory): one CTA per (node, group of 2-4
 *     samples) stages the node's matrix in shared memory and iterates the
 *     group's samples together (per-sample scalars, stopping tests and counts);
 *   AUTO: the library's choice. */
/* grf_options.timing: time only the phases of the mask in bits 0-7 (bit p is
 * grf_stats.phase_ms[p]); each timed phase adds two event records to the call */
#define GRF_TIMING_ONLY (1 << 30)

#define GRF_PCG_AUTO 0
#define GRF_PCG_PER_SYSTEM 1
#define GRF_PCG_STAGED 2
#define GRF_PCG_STAGED_PAIRS 3  /* as STAGED with 256-thread CTAs and groups of 2 samples:
                                   more resident CTAs per SM, half the matrix reuse */
#define GRF_PCG_BATCHED 4       /* mixed precision, Jacobi: one CTA per (node, 8 samples)
                                   with the group's vectors in global memory as rows of 8
                                   samples per vertex; what STAGED and STAGED_PAIRS fall
                                   back to when a node's system does not fit on chip */

typedef struct grf_stats {
  int64_t n_dofs;          /* N = |V_kept| + sum_e (n_e - 1) */
  int64_t n_nodes;         /* quadrature nodes solved (plus 1 per integer power) */
  int64_t n_systems;       /* vertex systems solved: nodes x samples */
  int64_t pcg_iters_total; /* sum of PCG iterations over all systems */
  int32_t pcg_iters_max;
  int32_t n_unconverged;   /* systems that hit max_iter */
  int32_t numeric_flag;    /* nonzero: NaN/Inf or p.Sp <= 0 met */
  int32_t kernel_launches; /* kernels this call launched */
  int32_t n_precond_fallback; /* systems whose learned preconditioner broke down
                                 (r.z <= 0 or p.Sp <= 0) and that finished with Jacobi */
  int32_t reserved;
  /* with grf_options.timing: device milliseconds per phase, measured with CUDA
   * events on the call's stream: [0] noise, [1] Schur blocks, [2] condensed
   * right-hand side, [3] vertex PCG, [4] recovery + quadrature sum,
   * [5] layout/mass scaling between stages, [6] learned-preconditioner network,
   * [7] unused; zero for the phases outside a GRF_TIMING_ONLY mask, and
   * without timing. With use_graph the events are nodes of the replayed graph
   * and the times are this call's replay. */
  double phase_ms[8];
} grf_stats;

/* Build a metric graph and its uniform mesh (Sec. 2.1 graph; Sec. 3, Phase 1
 * mesh: n_e = ceil(l_e / h), h_e = l_e / n_e).
 *   n_vertices >= 1, n_edges >= 1; edge_u/edge_v: host int64 [n_edges], ids in
 *   [0, n_vertices), no self-loops (parallel edges are allowed); lengths: host
 *   double [n_edges], finite and > 0; n_elems: host int32 [n_edges] with every
 *   entry >= 1, or NULL to use ceil(l_e / h) with h > 0.
 *   Degree-0 vertices are dropped (their lumped mass is 0).
 *   On success *out holds a new handle. Host-only; no device work. */
int grf_graph_create(int64_t n_vertices, int64_t n_edges, const int64_t* edge_u,
                     const int64_t* edge_v, const double* lengths,
                     const int32_t* n_elems, double h, grf_graph** out);

/* Release the handle and all device memory it cached. NULL is accepted. */
int grf_graph_destroy(grf_graph* g);

/* Sizes of the mesh (Sec. 3, Phase 1). Any output pointer may be NULL.
 *   vertex_map: host int64 [n_vertices input], input id -> kept id or -1.
 *   interior_offsets: host int64 [n_edges + 1]; the interior nodes of edge e
 *   are DOFs n_kept + interior_offsets[e] .. n_kept + interior_offsets[e+1]-1. */
int grf_graph_info(const grf_graph* g, int64_t* n_dofs, int64_t* n_kept_vertices,
                   int64_t* n_interior, int64_t* vertex_map, int64_t* interior_offsets);

/* The order in which the sample-group vertex PCG (Sec. 3, Phase 4) stores a
 * system in shared memory: reverse Cuthill-McKee, each connected component
 * in a contiguous range of slots (a launch detail: results do not depend on it).
 *   perm_out: host int64 [n_kept_vertices], slot i -> kept vertex id.
 *   GRF_EINVAL on a NULL handle or output. Host-only; no device work. */
int grf_graph_vertex_order(const grf_graph* g, int64_t* perm_out);

/* Draw n_samples fields of (kappa^2 - Delta)^beta u = W (Eq. 1) by the
 * lumped-mass, domain-decomposed sinc quadrature (Eq. 4, Eq. spde_approx_fem,
 * Sec. 3 Phases 2-5).
 *   kappa > 0; beta > 0; k_step > 0 (quadrature step); seed: Philox key.
 *   out: device buffer [n_samples][n_dofs] of double (GRF_OUT_F64) or float.
 *   opts: NULL for defaults. stream: cudaStream_t or NULL.
 *   stats: host, may be NULL. The call synchronises `stream` before returning.
 * Returns GRF_ENOCONV if some PCG hit max_iter (output still written),
 * GRF_ENUMERIC on NaN/Inf. */
int grf_sample(grf_graph* g, double kappa, double beta, double k_step, uint64_t seed,
               int64_t n_samples, void* out, const grf_options* opts, void* stream,
               grf_stats* stats);

/* The same through host memory: out_host is a host buffer of the layout above;
 * the call copies the field device -> host. For callers without device buffers.
 * The device-side output is a buffer cached on the handle (grown when needed),
 * so grf_options.use_graph replays stay valid across calls. */
int grf_sample_host(grf_graph* g, double kappa, double beta, double k_step, uint64_t seed,
                    int64_t n_samples, void* out_host, const grf_options* opts,
                    void* stream, grf_stats* stats);

/* n_calls draws of grf_sample_host (seeds[c], n_samples each) into the host
 * buffers out_host[c], pipelined: while call c computes on `stream`, the
 * field of call c - 1 crosses to the host on a second stream of the handle.
 * Each finished field is first copied device -> device into a second cached
 * device buffer (so that the next call, whose replayed CUDA graph writes the
 * first one, can start at once); every out_host[c] has the layout of
 * grf_sample. The copies run in call order on one stream, so entries may
 * repeat a buffer (the last call's field is what it holds). Pinned host
 * memory keeps the copies asynchronous. The results equal n_calls separate
 * grf_sample_host calls with the same seeds. Returns after the last copy;
 * stats (may be NULL) sums the calls' iteration counts and keeps the worst
 * status. Errors as grf_sample; GRF_EINVAL for n_calls < 0 or NULL arrays. */
int grf_sample_host_stream(grf_graph* g, double kappa, double beta, double k_step,
                           const uint64_t* seeds, int64_t n_calls, int64_t n_samples,
                           void* const* out_host, const grf_options* opts, void* stream,
                           grf_stats* stats);

/* White noise only (Eq. wh_def with the lumped factor, Sec. 2.5):
 *   raw_words != 0: out is uint32 [n_samples][n_dofs], word j of sample s =
 *     word (j mod 4) of Philox4x32-10(key = (seed lo32, seed hi32),
 *     counter = (q lo32, q hi32, s, 0)), q = j div 4;
 *   raw_words == 0: out is double [n_samples][n_dofs], b = sqrt(M_L) xi with
 *     u = (word + 1/2) 2^-32 and Box-Muller on the word pairs (0,1), (2,3):
 *     xi_a = sqrt(-2 ln u_a) cos(2 pi u_b), xi_b = sqrt(-2 ln u_a) sin(2 pi u_b);
 *   raw_words == 2: out is double [n_samples][n_dofs], the consistent-mass
 *     noise W = R xi (see GRF_MASS_CONSISTENT; computed in FP32; at most 256
 *     samples; uses the handle's workspace and synchronises nothing).
 * Asynchronous on `stream`. */
int grf_noise(grf_graph* g, uint64_t seed, int64_t n_samples, void* out, int32_t raw_words,
              void* stream);

/* General right-hand side: out = sum_l weight[l] (alpha[l] M_L + gamma[l] K)^{-1} rhs
 * through the same domain decomposition (Sec. 2.7 and Sec. 3, Phases 3-5).
 *   alpha >= 0, gamma > 0, weight: host double [n_nodes];
 *   rhs: device double [n_rhs][n_dofs]; out: device [n_rhs][n_dofs] per opts->out_dtype.
 *   Synchronises `stream`. */
int grf_apply(grf_graph* g, double kappa, int64_t n_nodes, const double* alpha,
              const double* gamma, const double* weight, int64_t n_rhs, const double* rhs,
              void* out, const grf_options* opts, void* stream, grf_stats* stats);

/* Vertex Schur system of one shifted matrix A = alpha M_L + gamma K (Eq.
 * global_schur, Eq. local_reduced_schur): S = sum_e S^(e) assembled from
 * per-edge 2x2 blocks.
 *   diag: device double [n_kept]   (S_vv);
 *   offdiag: device double [n_edges] (the coupling S_uv contributed by edge e).
 * Asynchronous on `stream`. */
int grf_schur(grf_graph* g, double kappa, double alpha, double gamma, double* diag,
              double* offdiag, void* stream);

/* Condensed right-hand side and vertex solution of one shifted system
 * (Eq. global_schur, Eq. local_reduced_schur, Phase 4 PCG):
 *   g_out[s][v] = rhs_v - sum_e A_vI^(e) (A_II^(e))^{-1} rhs_I^(e),
 *   u_out[s][v] solves S u = g by Jacobi-PCG.
 *   rhs: device double [n_rhs][n_dofs]; g_out, u_out: device double [n_rhs][n_kept].
 *   Synchronises `stream`. */
int grf_vertex_solve(grf_graph* g, double kappa, double alpha, double gamma, int64_t n_rhs,
                     const double* rhs, double* g_out, double* u_out,
                     const grf_options* opts, void* stream, grf_stats* stats);

/* grf_vertex_solve for callers that cannot allocate device memory: code whose
 * device memory is owned by another allocator with a fixed budget, or loops
 * that must not pay the device-wide synchronisation cudaMalloc/cudaFree can
 * cause. It allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine); all of its scratch lives in one static device array of 16 MiB that
 * every GPU loading this library holds until the process exits. The paper has
 * no counterpart to this entry point.
 *   Same arguments, layouts and results as grf_vertex_solve.
 *   The graph must already be resident on the current device: a call that may
 *   allocate (grf_vertex_solve, grf_sample, grf_noise, ...) must have used the
 *   graph on that device before; otherwise GRF_EINVAL, with no device work.
 *   Sizes whose scratch (about 8 n_dofs n_rhs bytes in FP64, 4 in mixed
 *   precision, plus the Schur system, the per-edge sweep constants and four
 *   PCG vectors per right-hand side; in mixed precision also the Schur system
 *   as FP32 pairs and four more vectors for the batched PCG's refinement)
 *   exceeds 16 MiB are rejected with GRF_EINVAL and a message naming the
 *   limit and the bytes needed.
 *   The first call on a device looks up the device address of the static array
 *   (once per device, with that device current); make that first call before
 *   any stream capture. All calls share the one array and it keeps the last
 *   call's contents: calls that overlap on the GPU (other streams, other
 *   threads) race with each other. grf_options.timing is ignored.
 *   Synchronises `stream`. */
int grf_vertex_solve_noalloc(grf_graph* g, double kappa, double alpha, double gamma,
                             int64_t n_rhs, const double* rhs, double* g_out, double* u_out,
                             const grf_options* opts, void* stream, grf_stats* stats);

/* Launch-schedule autotuner (the paper has no counterpart; it picks GPU launch
 * knobs only and does not change the computed field beyond rounding): times
 * grf_sample with CUDA events on `stream`, after one warm-up call each and
 * `reps` timed calls each, in three passes: first the edge-interior solvers
 * (mixed precision: THOMAS and SPECTRAL with recover_sg in {1, 2, 4} where
 * tridiagonal edges remain, SPECTRAL_TC, and SPECTRAL_UMMA for n_samples <= 256;
 * FP64: THOMAS) with the default PCG layout, then every PCG layout (PER_SYSTEM,
 * and in mixed precision STAGED, STAGED_PAIRS, BATCHED) with the fastest solver,
 * then, in mixed precision where FP32 tridiagonal edges remain, the sweep
 * layouts SEGMENTS and NODES against base->sweep (the segment/node split by
 * edge length).
 *   out: device buffer [n_samples][n_dofs] of base->out_dtype for the trials;
 *   base: options whose precision, out_dtype, rtol and max_iter are kept (NULL:
 *     defaults); best: receives base with the fastest knobs; best_ms: its mean
 *     milliseconds per call (may be NULL).
 * Synchronises `stream`. */
int grf_autotune(grf_graph* g, double kappa, double beta, double k_step, int64_t n_samples,
                 void* out, const grf_options* base, void* stream, int32_t reps,
                 grf_options* best, double* best_ms);

/* ---- Learned B B^T preconditioner of the vertex Schur systems (Phase 4).
 * An extension: the paper's own vertex PCG uses a Neumann-Neumann
 * preconditioner (Sec. 3, Phase 4, Neumann step). This one acts on the
 * Jacobi-scaled system S_hat = D^-1/2 S D^-1/2 (unit diagonal, off-diagonal
 * o_k = S^(e)_vw / sqrt(D_v D_w) for incidence k: vertex v, edge e, other end w;
 * a_k = -o_k >= 0):
 *   P = B B^T,  B = diag(exp(s)) + N,  N_{v w} = n_k on the incidence pattern,
 * so P is symmetric positive semi-definite and linear in the residual and
 * plain PCG stays valid. s and n come from a message-passing network whose
 * weights are shared by all nodes and graphs:
 *   x_v = [1, log(1+deg v)/3, sig_v, amax_v, sig_v^2, tanh(log(gamma/alpha)/20),
 *          sig_v/deg_v, 0],  sig_v = sum_k a_k,  amax_v = max_k a_k;
 *   h0 = relu(x W0 + b0);  h_i = relu([h_{i-1}, m_i] W_i + b_i),
 *   m_i(v) = sum_k a_k h_{i-1}(w_k),  i = 1..3 (width 64);
 *   s_v = h3_v . ws + cs;  n_k = a_k (h3_v . u + h3_w . up + cn).
 * Flat FP32 parameter vector (GRF_LP_PARAMS floats): W0 [8][64], b0 [64], then
 * W_i [128][64], b_i [64] for i = 1..3, then ws [64], cs, u [64], up [64], cn.
 * Matrices are row-major with the input index first. The dense layers run on
 * the tensor cores with BF16 operands and FP32 accumulation.
 * With the four heads (ws, cs, u/up, cn) at zero, B = I: exactly Jacobi.
 * Training loss over pairs (r, e) with S_hat e = r:
 *   mean over pairs of (P r - e)^T S_hat (P r - e) / (r^T e).
 * The weights live on the graph handle (device memory of its device). */
#define GRF_LP_PARAMS 25538

/* He-scaled random layers (normal, std sqrt(2 / fan_in), from `seed`) and zero
 * heads; resets the optimiser state. */
int grf_precond_init(grf_graph* g, uint64_t seed);

/* Copy the FP32 parameters in (host [n], n == GRF_LP_PARAMS) / out. set resets
 * the optimiser state. get fails if no weights have been set. */
int grf_precond_set(grf_graph* g, const float* params, int64_t n);
int grf_precond_get(const grf_graph* g, float* params, int64_t n);

/* Weights file: 48-byte little-endian header ("GRFLPBB1", version 1,
 * GRF_LP_PARAMS, 8 features, width 64, 3 layers, feature set 1, zeros) then
 * the FP32 parameter vector. load checks every header field. */
int grf_precond_save(const grf_graph* g, const char* path);
int grf_precond_load(grf_graph* g, const char* path);

/* Network output for one shifted system A = alpha M_L + gamma K (alpha > 0):
 *   s_out: host float [n_kept] (s_v), n_out: host float [2 n_edges] (n_k, in
 *   vertex-incidence order: vertices in kept order, each vertex's edges in
 *   increasing edge id). Either may be NULL. Synchronises `stream`. */
int grf_precond_forward(grf_graph* g, double kappa, double alpha, double gamma, float* s_out,
                        float* n_out, void* stream);

/* Training loss and its gradient for one shifted system and n_pairs given pairs:
 *   R, E: host float [n_pairs][n_kept] (r and e with S_hat e = r, e in the
 *   scaled unknowns); loss: host double; grad: host float [GRF_LP_PARAMS]
 *   (either may be NULL). Does not touch the optimiser state. Synchronises. */
int grf_precond_loss_grad(grf_graph* g, double kappa, double alpha, double gamma,
                          int64_t n_pairs, const float* R, const float* E, double* loss,
                          float* grad, void* stream);

typedef struct grf_train_options {
  int32_t epochs;           /* passes over the training nodes; <= 0: 40 */
  int32_t nodes_per_batch;  /* quadrature nodes per optimiser step; <= 0: 8 */
  int32_t n_samples;        /* white-noise right-hand sides per node; <= 0: 8 */
  int32_t pairs_per_system; /* (r, e) records per system; <= 0: 16 */
  int32_t record_stride;    /* CG iterations between records; <= 0: 2 */
  int32_t max_iter;         /* CG cap of the pair generation; <= 0: 4000 */
  double rtol;              /* CG stop of the pair generation; <= 0: 1e-10 */
  double lr;                /* Adam step; <= 0: 1e-3 */
  uint64_t seed;            /* noise seed and batch order */
} grf_train_options;

/* Train the network on this graph (weights must exist: init/set/load first).
 * Pairs: for every node of the sample call (kappa, beta, k_step) -- the
 * quadrature nodes, plus the stiffness node when beta >= 1 -- and n_samples
 * condensed white-noise right-hand sides, plain FP64 CG on S_hat records
 * r_i / ||r_i|| and e_i = (x* - x_i) / ||r_i|| every record_stride iterations
 * (x* = the converged iterate). Then Adam over random batches of nodes.
 *   loss_history: host float [epochs], mean batch loss per epoch (may be NULL);
 *   n_pairs: host, pairs recorded (may be NULL). Synchronises `stream`. */
int grf_precond_train(grf_graph* g, double kappa, double beta, double k_step,
                      const grf_train_options* opts, float* loss_history, int64_t* n_pairs,
                      void* stream);

/* Bytes of device workspace grf_sample would cache for this graph and size. */
int grf_workspace_bytes(const grf_graph* g, double beta, double k_step, int64_t n_samples,
                        const grf_options* opts, size_t* bytes);

/* Message of the last failed call on this thread ("" if none). */
const char* grf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GRF_H */
