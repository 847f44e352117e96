// Internal declarations shared by the sampler's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace grf {

// Device copy of the mesh (Sec. 3, Phase 1). Vertex ids are kept ids.
struct DevGraph {
  int32_t nv;        // kept vertices
  int32_t ne;        // edges
  int64_t ni;        // interior nodes
  int64_t n;         // DOFs = nv + ni
  const int32_t* eu;     // [ne] endpoint at x = 0
  const int32_t* ev;     // [ne] endpoint at x = l_e
  const int32_t* nel;    // [ne] elements n_e (>= 1)
  const double* he;      // [ne] element size h_e
  const int64_t* ioff;   // [ne + 1] interior offsets
  const int32_t* vptr;   // [nv + 1] vertex -> incidence list
  const int32_t* adj_edge;  // [2 ne] incident edge
  const int32_t* adj_nbr;   // [2 ne] vertex at the other end
  const double* sqrt_ml;    // [n] sqrt of the lumped mass per DOF
};

// Per-call node list: A_l = alpha_l M_L + gamma_l K, weight w_l.
struct DevNodes {
  int32_t L;
  const double* alpha;
  const double* gamma;
  const double* weight;
};

struct PcgStatus {
  int32_t n_unconverged;
  int32_t numeric_flag;
  int32_t iters_max;
  int32_t pad;
  unsigned long long iters_total;
};

// ---- noise.cu
// b[j][s] (sample-minor, T = float or double) = sqrt(M_L,j) xi_{s,j}
template <typename T>
void launch_noise_minor(const DevGraph& g, uint64_t seed, int64_t S, T* b, cudaStream_t st);
// sample-major output: raw words (uint32) or b in double
void launch_noise_major(const DevGraph& g, uint64_t seed, int64_t S, void* out, bool raw,
                        cudaStream_t st);

// ---- schur.cu
// Per-(l, e) 2x2 Schur blocks and vertex diagonal:
//   saa[l][e], sab[l][e];  diag[l][v] = sum_{e at v} saa[l][e];
//   offv[l][k] = sab[l][adj_edge[k]] in vertex-incidence order.
void launch_schur(const DevGraph& g, const DevNodes& nd, double kappa2, double* saa,
                  double* sab, double* diag, double* offv, cudaStream_t st);

// ---- thomas.cu
// rhs (sample-minor [n][S], T) -> condensed right-hand side gvec[l][s][v] (double)
template <typename T>
void launch_condense(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S,
                     const T* b, double* gvec, cudaStream_t st);
// Vertex accumulation out[s][v] = sum_l w_l x[l][s][v], and fused interior
// recovery + quadrature sum for the interior DOFs.
template <typename T, typename OutT>
void launch_recover(const DevGraph& g, const DevNodes& nd, double kappa2, int64_t S,
                    const T* b, const double* xv, OutT* out, double* acc, T* yscr, T* rpscr,
                    cudaStream_t st);
// [S][n] double -> [n][S] T, each DOF j scaled by scale[j] (or 1 when scale is null
// and mass_scale is false; by M_L,j = sqrt_ml[j]^2 when mass_scale is true)
template <typename T>
void launch_to_minor(const DevGraph& g, int64_t S, const double* src, T* dst, bool mass_scale,
                     cudaStream_t st);

// ---- pcg.cu
void launch_pcg_jacobi(const DevGraph& g, int32_t L, int64_t S, const double* diag,
                       const double* offv, const double* gvec, double* x, double* r, double* p,
                       double* q, double rtol, int32_t max_iter, int32_t* iters,
                       PcgStatus* status, cudaStream_t st);

int recover_sample_group();

}  // namespace grf
