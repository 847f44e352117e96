"""The sampled field by global sparse direct solves. Test infrastructure only.

U = sum_{l=-K^-}^{K^+} w_l (M_L + t_l K)^{-1} b,  K = kappa^2 M_L + G,
b = M_L^{1/2} xi (Eq. spde_approx_fem with the coefficients of Eq. 4; the
operator L = kappa^2 - Delta of Eq. 1 discretised with the lumped mass in both
the identity and the kappa^2 term). Each shifted matrix is factorised globally
by scipy's sparse LU (a library primitive standing for "solve"); nothing here
uses the edge/vertex splitting.

beta >= 1 (outside the paper's range (1/4, 1)): with beta = n + f, 0 < f < 1,
U = (K^{-1} M_L)^n U_f where U_f is the quadrature result for f; for an
integer beta = n, U = (K^{-1} M_L)^{n-1} K^{-1} b. (The discrete operator is
L_h = M_L^{-1} K, and L_h^{-beta} M_L^{-1} b is the FEM field.)
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, noise, quadrature


def assemble(mesh: fem.Mesh, kappa: float):
    ml = fem.lumped_mass(mesh)
    g = fem.stiffness(mesh)
    k = (kappa * kappa) * sp.diags(ml) + g
    return ml, g, k.tocsc()


def shifted_sum(ml: np.ndarray, kmat, b: np.ndarray, t, w) -> np.ndarray:
    """sum_l w_l (M_L + t_l K)^{-1} b for b of shape [S, N]."""
    out = np.zeros_like(b)
    mld = sp.diags(ml)
    for tl, wl in zip(t, w):
        lu = spla.splu((mld + tl * kmat).tocsc())
        out += wl * lu.solve(np.ascontiguousarray(b.T)).T
    return out


def stiff_solve(kmat, b: np.ndarray) -> np.ndarray:
    return spla.splu(kmat.tocsc()).solve(np.ascontiguousarray(b.T)).T


def fractional_apply(ml, kmat, b, beta: float, k: float) -> np.ndarray:
    n_int = math.floor(beta)
    frac = beta - n_int
    if frac < 1e-12:
        u = stiff_solve(kmat, b)
        reps = n_int - 1
    else:
        t, w = quadrature.nodes(frac, k)
        u = shifted_sum(ml, kmat, b, t, w)
        reps = n_int
    for _ in range(reps):
        u = stiff_solve(kmat, ml[None, :] * u)
    return u


def sample(graph, kappa: float, beta: float, k: float, seed: int, n_samples: int,
           h: float | None = None, n_elems=None, clip=None):
    """Returns (mesh, U [S, N], b [S, N])."""
    mesh = fem.build_mesh(graph.edge_u, graph.edge_v, graph.lengths,
                          graph.n_vertices, h=h, n_elems=n_elems, clip=clip)
    ml, _, kmat = assemble(mesh, kappa)
    b = noise.white_noise(ml, seed, n_samples)
    return mesh, fractional_apply(ml, kmat, b, beta, k), b


def vertex_condensation(mesh: fem.Mesh, ml, kmat, t: float, b: np.ndarray,
                        alpha: float = 1.0):
    """For A = alpha M_L + t K split into vertex (G) and interior (I) blocks:
    the condensed right-hand side g = b_G - A_GI A_II^{-1} b_I and the vertex
    values u_G of A^{-1} b (Eq. global_schur). b: [S, N]. Used to check the
    intermediate vectors of a split solver; computed from the global blocks."""
    nv = mesh.n_vertices
    a = (alpha * sp.diags(ml) + t * kmat).tocsr()
    a_gi = a[:nv, nv:]
    a_ii = a[nv:, nv:].tocsc()
    bt = np.ascontiguousarray(b.T)
    if mesh.n_interior:
        w = spla.splu(a_ii).solve(np.ascontiguousarray(bt[nv:]))
        g = bt[:nv] - a_gi @ w
    else:
        g = bt[:nv].copy()
    u = spla.splu(a.tocsc()).solve(bt)
    return g.T, u[:nv].T


def edge_schur_blocks(mesh: fem.Mesh, kappa: float, t: float, alpha: float = 1.0):
    """Per-edge 2x2 Schur blocks (Eq. local_reduced_schur) of A = alpha M_L + t K
    by dense elimination of each edge's own element-assembled matrix: returns
    (s_uu [E], s_uv [E]); the blocks are symmetric with s_vv = s_uu on a uniform
    edge mesh. Small meshes only."""
    E = mesh.edge_u.shape[0]
    suu = np.zeros(E)
    suv = np.zeros(E)
    for e in range(E):
        n, h = int(mesh.n_elems[e]), float(mesh.h_e[e])
        a = np.zeros((n + 1, n + 1))
        for k in range(n):
            idx = [k, k + 1]
            a[np.ix_(idx, idx)] += (alpha + t * kappa ** 2) * h / 2 * np.eye(2) + \
                t / h * np.array([[1.0, -1.0], [-1.0, 1.0]])
        bnd = [0, n]
        inn = list(range(1, n))
        s = a[np.ix_(bnd, bnd)]
        if inn:
            s = s - a[np.ix_(bnd, inn)] @ np.linalg.solve(a[np.ix_(inn, inn)], a[np.ix_(inn, bnd)])
        suu[e], suv[e] = s[0, 0], s[0, 1]
    return suu, suv


def vertex_schur_dense(mesh: fem.Mesh, ml, kmat, t: float, alpha: float = 1.0):
    """S = A_GG - A_GI A_II^{-1} A_IG as a dense |V| x |V| matrix (small graphs)."""
    nv = mesh.n_vertices
    a = (alpha * sp.diags(ml) + t * kmat).tocsr()
    s = a[:nv, :nv].toarray()
    if mesh.n_interior:
        a_ig = a[nv:, :nv].toarray()
        z = spla.splu(a[nv:, nv:].tocsc()).solve(a_ig)
        s = s - a[:nv, nv:] @ z
    return s
