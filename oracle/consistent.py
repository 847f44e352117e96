"""The consistent-mass comparison system (Sec. 2.4 Eq. wh_def, Sec. 3 Phase 2
consistent case): white noise W = R xi with M = R R^T the Cholesky factor of
the consistent mass matrix, and the shifted systems with the consistent mass
in the operator, U = sum_l w_l (M + t_l K_c)^{-1} W, K_c = kappa^2 M + G.
Test infrastructure only (see package header).

Consistent mass (Sec. 3 Phase 2): 2h/3 and h/6 on and beside the diagonal of
an edge interior, sum h_e/3 at a vertex, h_e/6 between a vertex and its
adjacent interior node (assembled here from the element matrix
h/6 [[2, 1], [1, 2]]).

Reading (the paper does not fix the order of the factorisation): R is the
lower Cholesky factor of M with the DOFs in the order of the partition of
Phase 2, the interior nodes edge by edge (each edge from edge_u towards
edge_v) and then the vertices by kept id; xi_j is the standard normal of DOF j
(the Philox stream of noise.py) and W_j is the entry of R xi for DOF j.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, noise, quadrature


def cholesky_order(mesh: fem.Mesh) -> np.ndarray:
    """DOFs in elimination order: interiors (edge by edge), then vertices."""
    return np.concatenate([np.arange(mesh.n_vertices, mesh.n_dofs),
                           np.arange(mesh.n_vertices)])


def cholesky_factor(mesh: fem.Mesh) -> np.ndarray:
    """Dense lower Cholesky factor of the consistent mass in elimination order
    (small meshes only)."""
    perm = cholesky_order(mesh)
    m = fem.consistent_mass(mesh).toarray()[np.ix_(perm, perm)]
    return np.linalg.cholesky(m)


def white_noise(mesh: fem.Mesh, seed: int, n_samples: int) -> np.ndarray:
    """W = R xi, shape [n_samples, n_dofs] in DOF order."""
    perm = cholesky_order(mesh)
    xi = noise.standard_normals(seed, mesh.n_dofs, n_samples)
    r = cholesky_factor(mesh)
    w = np.empty_like(xi)
    w[:, perm] = (r @ xi[:, perm].T).T
    return w


def assemble(mesh: fem.Mesh, kappa: float):
    mc = fem.consistent_mass(mesh)
    g = fem.stiffness(mesh)
    return mc.tocsc(), g, ((kappa * kappa) * mc + g).tocsc()


def fractional_apply(mc, kc, b: np.ndarray, beta: float, k: float) -> np.ndarray:
    """(M^{-1} K_c)^{-beta} M^{-1} b by the quadrature of Eq. 4 for the
    fractional part and stiffness solves (K_c^{-1} M)^n for the integer part."""
    n_int = math.floor(beta)
    frac = beta - n_int
    if frac < 1e-12:
        u = spla.splu(kc.tocsc()).solve(np.ascontiguousarray(b.T)).T
        reps = n_int - 1
    else:
        t, w = quadrature.nodes(frac, k)
        u = np.zeros_like(b)
        for tl, wl in zip(t, w):
            lu = spla.splu((mc + tl * kc).tocsc())
            u += wl * lu.solve(np.ascontiguousarray(b.T)).T
        reps = n_int
    lu_k = spla.splu(kc.tocsc()) if reps > 0 else None
    for _ in range(reps):
        u = lu_k.solve(np.ascontiguousarray((mc @ u.T))).T
    return u


def sample(graph, kappa: float, beta: float, k: float, seed: int, n_samples: int,
           h: float | None = None, n_elems=None):
    """Returns (mesh, U [S, N], W [S, N]) of the consistent-mass sampler."""
    mesh = fem.build_mesh(graph.edge_u, graph.edge_v, graph.lengths, graph.n_vertices,
                          h=h, n_elems=n_elems)
    mc, _, kc = assemble(mesh, kappa)
    w = white_noise(mesh, seed, n_samples)
    return mesh, fractional_apply(mc, kc, w, beta, k), w


def interval_closed_form(n: int, length: float, kappa: float, beta: float, k: float,
                         w: np.ndarray) -> np.ndarray:
    """On one interval (Kirchhoff = Neumann ends) with n uniform elements the
    consistent-mass P1 pencil (G, M) has the eigenvectors v_j(i) = cos(j pi i / n)
    (positions i = 0..n) and eigenvalues
    lambda_j = 6 (1 - cos(j pi / n)) / (h^2 (2 + cos(j pi / n))); hence
    U = sum_j q(kappa^2 + lambda_j) (v_j . W) / (v_j^T M v_j) v_j with q the
    scalar quadrature. w: [S, n + 1] by position along the interval."""
    h = length / n
    i = np.arange(n + 1)
    out = np.zeros_like(w)
    mpos = np.zeros((n + 1, n + 1))
    for a in range(n):
        mpos[a:a + 2, a:a + 2] += h / 6 * np.array([[2.0, 1.0], [1.0, 2.0]])
    for j in range(n + 1):
        v = np.cos(j * math.pi * i / n)
        lam = 6.0 * (1.0 - math.cos(j * math.pi / n)) / (h * h * (2.0 + math.cos(j * math.pi / n)))
        q = float(quadrature.scalar(np.array([kappa * kappa + lam]), beta, k)[0])
        nu = float(v @ mpos @ v)
        out += q * np.outer(w @ v, v) / nu
    return out
