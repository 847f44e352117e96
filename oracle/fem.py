"""Mesh, DOF map, lumped mass and P1 stiffness of a metric graph, assembled
element by element over the whole graph. Test infrastructure only (see
package header).

Mesh (Sec. 3, Phase 1): edge e of length l_e gets n_e = ceil(l_e / h) uniform
elements of size h_e = l_e / n_e (or a caller-given n_e), hence n_e - 1
interior nodes.

DOF order: the kept vertices first (degree-0 vertices are dropped: their
lumped mass is zero and the shifted systems would be singular), then the
interior nodes edge by edge, each edge from edge_u towards edge_v.

Lumped mass (Sec. 3, Phase 2, lumped case): row sums of the consistent mass,
h_e on interior nodes and sum_{e at v} h_e / 2 at a vertex. Assembled here as
h_e / 2 per element end point.

Stiffness (Sec. 3, Phase 2): 2/h_e and -1/h_e on interiors, sum 1/h_e at a
vertex, -1/h_e between a vertex and its adjacent interior node. Assembled here
as the element matrix [[1, -1], [-1, 1]] / h_e.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Mesh:
    n_vertices_in: int
    n_vertices: int          # kept vertices
    vertex_map: np.ndarray   # input id -> kept id or -1
    edge_u: np.ndarray       # kept ids
    edge_v: np.ndarray
    lengths: np.ndarray
    n_elems: np.ndarray      # int64 [E]
    h_e: np.ndarray          # float64 [E]
    interior_offsets: np.ndarray  # int64 [E+1], offsets into the interior block
    n_interior: int
    n_dofs: int


def build_mesh(edge_u, edge_v, lengths, n_vertices: int, h: float | None = None,
               n_elems=None, clip: tuple[int, int] | None = None) -> Mesh:
    edge_u = np.asarray(edge_u, np.int64)
    edge_v = np.asarray(edge_v, np.int64)
    lengths = np.asarray(lengths, np.float64)
    if np.any(edge_u == edge_v):
        raise ValueError("self-loop")
    if n_elems is None:
        n = np.ceil(lengths / h).astype(np.int64)
        if clip is not None:
            n = np.clip(n, clip[0], clip[1])
    else:
        n = np.asarray(n_elems, np.int64)
    n = np.maximum(n, 1)
    deg = np.bincount(np.concatenate([edge_u, edge_v]), minlength=n_vertices)
    kept = deg > 0
    vmap = -np.ones(n_vertices, np.int64)
    vmap[kept] = np.arange(int(kept.sum()))
    nv = int(kept.sum())
    offs = np.zeros(edge_u.shape[0] + 1, np.int64)
    offs[1:] = np.cumsum(n - 1)
    ni = int(offs[-1])
    return Mesh(n_vertices, nv, vmap, vmap[edge_u], vmap[edge_v], lengths, n,
                lengths / n, offs, ni, nv + ni)


def elements(m: Mesh):
    """All elements of the mesh as (dof_a, dof_b, h): element k of edge e joins
    position k and k+1 along the edge, position 0 being edge_u, position n_e
    being edge_v and position p in between being interior node p."""
    E = m.edge_u.shape[0]
    ne = m.n_elems
    eid = np.repeat(np.arange(E), ne)
    start = np.repeat(np.cumsum(ne) - ne, ne)
    k = np.arange(int(ne.sum())) - start

    def dof(pos):
        d = m.n_vertices + m.interior_offsets[eid] + pos - 1
        d = np.where(pos == 0, m.edge_u[eid], d)
        d = np.where(pos == ne[eid], m.edge_v[eid], d)
        return d

    return dof(k), dof(k + 1), m.h_e[eid]


def lumped_mass(m: Mesh) -> np.ndarray:
    a, b, h = elements(m)
    ml = np.zeros(m.n_dofs)
    np.add.at(ml, a, h / 2)
    np.add.at(ml, b, h / 2)
    return ml


def consistent_mass(m: Mesh) -> sp.csr_matrix:
    """Element mass h/6 [[2, 1], [1, 2]] (used only to pin the lumped mass as
    its row sums)."""
    a, b, h = elements(m)
    rows = np.concatenate([a, b, a, b])
    cols = np.concatenate([a, b, b, a])
    vals = np.concatenate([h / 3, h / 3, h / 6, h / 6])
    return sp.csr_matrix((vals, (rows, cols)), shape=(m.n_dofs, m.n_dofs))


def stiffness(m: Mesh) -> sp.csr_matrix:
    a, b, h = elements(m)
    rows = np.concatenate([a, b, a, b])
    cols = np.concatenate([a, b, b, a])
    vals = np.concatenate([1 / h, 1 / h, -1 / h, -1 / h])
    return sp.csr_matrix((vals, (rows, cols)), shape=(m.n_dofs, m.n_dofs))
