"""Convergence study of the lumped-mass sampler on the GPU (Sec. 4.1 strong
error, Sec. 4.2 covariance error, Table 1), through the C ABI.

Nested meshes: level q gives edge e n_e = base_e 2^q uniform elements (h_max
halves per level), so the coarse basis functions are combinations of the fine
ones through the linear interpolation P (coarse nodes -> fine nodes). Every
solve is grf_apply with the sinc nodes of Eq. 4 at the step k = -1/(beta ln h)
and the limits of Sec. 4.1 of that mesh; the noise is grf_noise on the
overkill mesh (W = M_L^{1/2} xi) and its projection to a coarse mesh is P^T W
(the integrals of the noise against the coarse basis functions). The host only
builds P, the consistent mass of the overkill mesh (the exact L2(Gamma) inner
product of piecewise-linear functions) and the error norms.

Strong error: root mean square over realizations of ||u_ok - P u_h||_L2(Gamma).
Covariance error: ||C_ok - P C_h P^T||_L2(Gamma x Gamma), C_h = Q_h M_L Q_h^T,
Q_h = sum_l w_l (M_L + t_l K)^{-1} (its columns from grf_apply on the columns
of M_L^{1/2}). Rates: least-squares slope of ln err against ln h.

    python -m paper_2605_02670_gb300.convergence   # prints a table like Table 1
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import Graph


def nested_graph(graph, base_counts, level: int) -> Graph:
    n = np.asarray(base_counts, np.int64) * (2 ** level)
    return Graph(graph.edge_u, graph.edge_v, graph.lengths, graph.n_vertices,
                 n_elems=n.astype(np.int32))


def _counts(base_counts, level):
    return np.asarray(base_counts, np.int64) * (2 ** level)


def _dof(G: Graph, ne, e: int, p: int) -> int:
    """DOF of position p (0 .. n_e) along edge e: the vertices first (kept ids),
    then the interior nodes edge by edge."""
    if p == 0:
        return int(G.vertex_map[G.edge_u_in[e]])
    if p == ne[e]:
        return int(G.vertex_map[G.edge_v_in[e]])
    return G.n_kept + int(G.interior_offsets[e]) + p - 1


def prolongation(Gc: Graph, nc, Gf: Graph, nf) -> sp.csr_matrix:
    """Linear interpolation from the coarse to the fine nodes, [N_f, N_c]."""
    rows, cols, vals = [], [], []
    for v in range(Gc.n_kept):
        rows.append(v)
        cols.append(v)
        vals.append(1.0)
    for e in range(len(nc)):
        r = int(nf[e] // nc[e])
        for q in range(1, int(nf[e])):
            fd = _dof(Gf, nf, e, q)
            a, t = divmod(q, r)
            if t == 0:
                rows.append(fd)
                cols.append(_dof(Gc, nc, e, a))
                vals.append(1.0)
            else:
                s = t / r
                rows += [fd, fd]
                cols += [_dof(Gc, nc, e, a), _dof(Gc, nc, e, a + 1)]
                vals += [1.0 - s, s]
    return sp.csr_matrix((vals, (rows, cols)), shape=(Gf.n_dofs, Gc.n_dofs))


def element_mass(G: Graph, lengths, ne, lumped: bool):
    """Consistent mass (sparse) or lumped mass (vector) of the mesh: element
    matrix h/6 [[2, 1], [1, 2]], lumped h/2 per element end."""
    a, b, hv = [], [], []
    for e in range(len(ne)):
        h = float(lengths[e]) / int(ne[e])
        for k in range(int(ne[e])):
            a.append(_dof(G, ne, e, k))
            b.append(_dof(G, ne, e, k + 1))
            hv.append(h)
    a, b, hv = np.array(a), np.array(b), np.array(hv)
    if lumped:
        ml = np.zeros(G.n_dofs)
        np.add.at(ml, a, hv / 2)
        np.add.at(ml, b, hv / 2)
        return ml
    rows = np.concatenate([a, b, a, b])
    cols = np.concatenate([a, b, b, a])
    vals = np.concatenate([hv / 3, hv / 3, hv / 6, hv / 6])
    return sp.csr_matrix((vals, (rows, cols)), shape=(G.n_dofs, G.n_dofs))


def sinc_nodes(beta: float, k: float):
    """(t_l, w_l) of Eq. 4 with the limits of Sec. 4.1 (0 < beta < 1)."""
    km = math.ceil(math.pi ** 2 / (4 * k * k * beta))
    kp = math.ceil(math.pi ** 2 / (4 * k * k * (1 - beta)))
    y = np.arange(-km, kp + 1, dtype=np.float64) * k
    return np.exp(2 * y), (2 * k * math.sin(math.pi * beta) / math.pi) * np.exp(2 * beta * y)


def fractional_apply(G: Graph, kappa: float, beta: float, h: float, rhs, precision: str):
    """L_h^{-beta} rhs (rhs [S, N] on the device) with k = -1/(beta ln h)."""
    t, w = sinc_nodes(beta, -1.0 / (beta * math.log(h)))
    out, _ = G.apply(kappa, np.ones_like(t), t, w, rhs, precision=precision, out_dtype="f64")
    return out


def strong_errors(graph, base_counts, levels, level_ok: int, beta: float, kappa: float,
                  n_real: int, seed: int, precision: str = "mixed"):
    import torch
    nf = _counts(base_counts, level_ok)
    Gf = nested_graph(graph, base_counts, level_ok)
    hf = float((np.asarray(graph.lengths) / nf).max())
    wf = Gf.noise(seed, n_real)  # [S, N_f] FP64 on the device
    uf = fractional_apply(Gf, kappa, beta, hf, wf, precision).cpu().numpy()
    wfh = wf.cpu().numpy()
    M = element_mass(Gf, graph.lengths, nf, lumped=False)
    hs, errs = [], []
    for q in levels:
        nc = _counts(base_counts, q)
        Gc = nested_graph(graph, base_counts, q)
        P = prolongation(Gc, nc, Gf, nf)
        wc = torch.tensor(np.ascontiguousarray((P.T @ wfh.T).T), device="cuda")
        hc = float((np.asarray(graph.lengths) / nc).max())
        uc = fractional_apply(Gc, kappa, beta, hc, wc, precision).cpu().numpy()
        d = uf - (P @ uc.T).T
        e2 = np.einsum("sn,sn->s", d, (M @ d.T).T)
        hs.append(hc)
        errs.append(math.sqrt(float(e2.mean())))
    return np.array(hs), np.array(errs)


def covariance(G: Graph, lengths, ne, kappa, beta, h, precision):
    import torch
    ml = element_mass(G, lengths, ne, lumped=True)
    y = fractional_apply(G, kappa, beta, h, torch.tensor(np.diag(np.sqrt(ml)), device="cuda"),
                         precision).cpu().numpy()
    return y.T @ y


def covariance_errors(graph, base_counts, levels, level_ok: int, beta: float, kappa: float,
                      precision: str = "mixed"):
    nf = _counts(base_counts, level_ok)
    Gf = nested_graph(graph, base_counts, level_ok)
    hf = float((np.asarray(graph.lengths) / nf).max())
    cf = covariance(Gf, graph.lengths, nf, kappa, beta, hf, precision)
    M = element_mass(Gf, graph.lengths, nf, lumped=False).toarray()
    hs, errs = [], []
    for q in levels:
        nc = _counts(base_counts, q)
        Gc = nested_graph(graph, base_counts, q)
        P = prolongation(Gc, nc, Gf, nf).toarray()
        hc = float((np.asarray(graph.lengths) / nc).max())
        d = cf - P @ covariance(Gc, graph.lengths, nc, kappa, beta, hc, precision) @ P.T
        hs.append(hc)
        errs.append(math.sqrt(max(float(np.trace(M @ d @ M @ d)), 0.0)))
    return np.array(hs), np.array(errs)


def rate(hs, errs) -> float:
    x = np.log(np.asarray(hs, np.float64))
    y = np.log(np.asarray(errs, np.float64))
    return float(np.polyfit(x, y, 1)[0])


def study_graph():
    """A small synthetic metric graph (the experiments' own graph is not
    available): a triangle of unit edges with a pendant edge of length 1/2."""
    from types import SimpleNamespace
    return (SimpleNamespace(n_vertices=4, edge_u=np.array([0, 1, 2, 2]),
                            edge_v=np.array([1, 2, 0, 3]),
                            lengths=np.array([1.0, 1.0, 1.0, 0.5])),
            np.array([2, 2, 2, 1]))


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--betas", default="0.375,0.5,0.625,0.75,0.875")
    ap.add_argument("--levels", default="2,3,4,5")  # h_max = 2^-3 .. 2^-6
    ap.add_argument("--level-ok", type=int, default=12)
    ap.add_argument("--level-ok-cov", type=int, default=8)
    ap.add_argument("--realizations", type=int, default=100)
    ap.add_argument("--precision", default="mixed")
    a = ap.parse_args()
    g, base = study_graph()
    levels = [int(x) for x in a.levels.split(",")]
    rows = []
    for beta in [float(x) for x in a.betas.split(",")]:
        hs, es = strong_errors(g, base, levels, a.level_ok, beta, 1.0, a.realizations, 1,
                               a.precision)
        hc, ec = covariance_errors(g, base, levels, a.level_ok_cov, beta, 1.0, a.precision)
        rows.append({"beta": beta, "h": hs.tolist(), "strong": es.tolist(),
                     "strong_rate": rate(hs, es), "strong_theory": 2 * beta - 0.5,
                     "cov": ec.tolist(), "cov_rate": rate(hc, ec),
                     "cov_theory": min(4 * beta - 0.5, 2.0)})
        print(json.dumps(rows[-1]), flush=True)


if __name__ == "__main__":
    main()
