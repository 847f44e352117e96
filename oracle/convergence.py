"""Convergence study of the lumped-mass method (Sec. 4.1 strong error, Sec. 4.2
covariance error, Table 1). Test infrastructure only (see package header).

Meshes are nested: level q gives every edge n_e = base_e 2^q uniform elements,
so h_max halves per level and every coarse basis function is a combination of
the fine ones, phi_i^c = sum_j P_ji phi_j^f with P the linear interpolation
(prolongation) from the coarse to the fine nodes.

Strong error (Sec. 4.1): white noise drawn on the overkill (finest) mesh as the
lumped-mass vector W_f = M_L^{1/2} xi; the coarse right-hand side is its
projection W_c = P^T W_f (W_i = integral of the noise against phi_i); the coarse
field U_c = L_h^{-beta} solve of Eq. spde_approx_fem with the quadrature of
Eq. 4, k = -1 / (beta ln h) and the limits of Sec. 4.1; the error
e = U_f - P U_c on the overkill mesh in the L2(Gamma) norm
e^T M e (M the consistent mass of the overkill mesh: the exact L2 norm of a
piecewise-linear function). The reported error is the root of the mean over
the realizations (the printed errors halve per halving of h at beta = 3/4,
i.e. they follow the rate 2 beta - 1/2 of the norm itself).

Covariance error (Sec. 4.2): the covariance of the method on mesh h is
C_h = Q_h M_L Q_h^T with Q_h = sum_l w_l (M_L + t_l K)^{-1}; the error is the
L2(Gamma x Gamma) norm of C_f - P C_h P^T for the piecewise-linear
representation, trace(M D M D) with D the difference and M the overkill mesh's
consistent mass.

Rates are the slopes of the least-squares line ln err = c + r ln h.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import fem, noise, sampler


def nested_mesh(graph, base_counts, level: int) -> fem.Mesh:
    n = np.asarray(base_counts, np.int64) * (2 ** level)
    return fem.build_mesh(graph.edge_u, graph.edge_v, graph.lengths, graph.n_vertices,
                          n_elems=n)


def h_max(mesh: fem.Mesh) -> float:
    return float(mesh.h_e.max())


def quad_step(beta: float, h: float) -> float:
    """k = -1 / (beta ln h) (Sec. 4.1)."""
    return -1.0 / (beta * math.log(h))


def prolongation(mc: fem.Mesh, mf: fem.Mesh) -> sp.csr_matrix:
    """Linear interpolation from the coarse nodes to the fine nodes of a nested
    pair (fine edge e has r_e = n_e^f / n_e^c elements per coarse element).
    Returns P with shape [N_f, N_c]."""
    rows, cols, vals = [], [], []
    for v in range(mc.n_vertices):  # vertices are shared
        rows.append(v)
        cols.append(v)
        vals.append(1.0)
    for e in range(mc.edge_u.shape[0]):
        nc, nf = int(mc.n_elems[e]), int(mf.n_elems[e])
        r = nf // nc
        assert nc * r == nf

        def cdof(p):  # coarse DOF of position p along the edge
            if p == 0:
                return int(mc.edge_u[e])
            if p == nc:
                return int(mc.edge_v[e])
            return mc.n_vertices + int(mc.interior_offsets[e]) + p - 1

        for q in range(1, nf):  # fine interior node q
            fd = mf.n_vertices + int(mf.interior_offsets[e]) + q - 1
            a, t = divmod(q, r)
            if t == 0:
                rows.append(fd)
                cols.append(cdof(a))
                vals.append(1.0)
            else:
                s = t / r
                rows += [fd, fd]
                cols += [cdof(a), cdof(a + 1)]
                vals += [1.0 - s, s]
    return sp.csr_matrix((vals, (rows, cols)), shape=(mf.n_dofs, mc.n_dofs))


def level_solve(mesh: fem.Mesh, kappa: float, beta: float, rhs: np.ndarray) -> np.ndarray:
    """L_h^{-beta} applied to the right-hand sides [S, N] of mesh h (Eq.
    spde_approx_fem with the step k of Sec. 4.1 for this mesh)."""
    ml, _, kmat = sampler.assemble(mesh, kappa)
    k = quad_step(beta, h_max(mesh))
    return sampler.fractional_apply(ml, kmat, rhs, beta, k)


def strong_errors(graph, base_counts, levels, level_ok: int, beta: float, kappa: float,
                  n_real: int, seed: int):
    """(h per level, root-mean-square L2 errors per level)."""
    mf = nested_mesh(graph, base_counts, level_ok)
    mlf = fem.lumped_mass(mf)
    wf = noise.white_noise(mlf, seed, n_real)
    uf = level_solve(mf, kappa, beta, wf)
    mcons = fem.consistent_mass(mf)
    hs, errs = [], []
    for q in levels:
        mc = nested_mesh(graph, base_counts, q)
        P = prolongation(mc, mf)
        wc = (P.T @ wf.T).T
        uc = level_solve(mc, kappa, beta, wc)
        d = uf - (P @ uc.T).T
        e2 = np.einsum("sn,sn->s", d, (mcons @ d.T).T)
        hs.append(h_max(mc))
        errs.append(math.sqrt(float(e2.mean())))
    return np.array(hs), np.array(errs)


def covariance(mesh: fem.Mesh, kappa: float, beta: float) -> np.ndarray:
    """C_h = Q_h M_L Q_h^T, dense (small meshes only)."""
    ml = fem.lumped_mass(mesh)
    y = level_solve(mesh, kappa, beta, np.diag(np.sqrt(ml)))  # rows: Q M_L^{1/2} columns
    return y.T @ y


def covariance_errors(graph, base_counts, levels, level_ok: int, beta: float, kappa: float):
    """(h per level, L2(Gamma x Gamma) errors per level)."""
    mf = nested_mesh(graph, base_counts, level_ok)
    cf = covariance(mf, kappa, beta)
    M = fem.consistent_mass(mf).toarray()
    hs, errs = [], []
    for q in levels:
        mc = nested_mesh(graph, base_counts, q)
        P = prolongation(mc, mf).toarray()
        d = cf - P @ covariance(mc, kappa, beta) @ P.T
        hs.append(h_max(mc))
        errs.append(math.sqrt(max(float(np.trace(M @ d @ M @ d)), 0.0)))
    return np.array(hs), np.array(errs)


def rate(hs, errs) -> float:
    """Slope r of the least-squares line ln err = c + r ln h."""
    x = np.log(np.asarray(hs, np.float64))
    y = np.log(np.asarray(errs, np.float64))
    return float(np.polyfit(x, y, 1)[0])
