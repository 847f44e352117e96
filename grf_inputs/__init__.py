"""Seeded synthetic graph workloads shared by the oracle, the tests and the bench.

This module only draws graphs (vertex/edge lists and edge lengths) and names the
sampling parameters of each workload. It holds none of the sampler's arithmetic:
no mesh, no mass or stiffness entries, no quadrature. Both the CPU oracle and the
CUDA path derive everything else from these lists on their own.

The graph families follow the workloads used for the method's experiments
(Sec. 4, performance comparison: Barabasi-Albert graphs) plus the synthetic
families used to exercise the GPU path: a small square-with-diagonal graph, a
random geometric graph, a Barabasi-Albert graph with log-normal lengths and a
grid with randomly deleted edges. The generators are written here with numpy so
that they run where networkx is absent; they are statistically the standard
models but not edge-for-edge identical to networkx's output.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Graph:
    n_vertices: int
    edge_u: np.ndarray  # int64 [E]
    edge_v: np.ndarray  # int64 [E]
    lengths: np.ndarray  # float64 [E]

    @property
    def n_edges(self) -> int:
        return int(self.edge_u.shape[0])


def square_diagonal(seed: int = 0) -> Graph:
    """Square 0-1-2-3-0 plus the diagonal 0-2; lengths U[0.5, 1.5]."""
    eu = np.array([0, 1, 2, 3, 0], dtype=np.int64)
    ev = np.array([1, 2, 3, 0, 2], dtype=np.int64)
    rng = np.random.default_rng(seed)
    lengths = rng.uniform(0.5, 1.5, size=5)
    return Graph(4, eu, ev, lengths)


def interval(length: float = 1.0) -> Graph:
    """A single edge between two degree-1 vertices."""
    return Graph(2, np.array([0], np.int64), np.array([1], np.int64),
                 np.array([float(length)]))


def random_geometric(n: int = 2000, radius: float = 0.0285, seed: int = 0,
                     length_scale: float = 10.0) -> Graph:
    """n points uniform in the unit square; an edge joins every pair closer
    than `radius`; edge length = length_scale * Euclidean distance.
    Isolated vertices are kept in the lists (the sampler drops them)."""
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, size=(n, 2))
    # cell grid to avoid the n^2 pair loop
    ncell = max(1, int(1.0 / radius))
    cell = np.minimum((pts / (1.0 / ncell)).astype(np.int64), ncell - 1)
    key = cell[:, 0] * ncell + cell[:, 1]
    order = np.argsort(key, kind="stable")
    buckets: dict[int, list[int]] = {}
    for idx in order:
        buckets.setdefault(int(key[idx]), []).append(int(idx))
    us, vs = [], []
    for cx in range(ncell):
        for cy in range(ncell):
            a = buckets.get(cx * ncell + cy)
            if not a:
                continue
            for dx in (0, 1):
                for dy in (-1, 0, 1):
                    if dx == 0 and dy < 0:
                        continue
                    nx_, ny_ = cx + dx, cy + dy
                    if not (0 <= nx_ < ncell and 0 <= ny_ < ncell):
                        continue
                    b = buckets.get(nx_ * ncell + ny_)
                    if not b:
                        continue
                    A = np.array(a)
                    B = np.array(b)
                    d = np.linalg.norm(pts[A][:, None, :] - pts[B][None, :, :], axis=2)
                    ii, jj = np.nonzero(d <= radius)
                    for i, j in zip(ii, jj):
                        u, v = int(A[i]), int(B[j])
                        if dx == 0 and dy == 0 and u >= v:
                            continue
                        us.append(min(u, v))
                        vs.append(max(u, v))
    eu = np.array(us, dtype=np.int64)
    ev = np.array(vs, dtype=np.int64)
    srt = np.lexsort((ev, eu))
    eu, ev = eu[srt], ev[srt]
    lengths = length_scale * np.linalg.norm(pts[eu] - pts[ev], axis=1)
    return Graph(n, eu, ev, lengths)


def barabasi_albert(n: int, m: int, seed: int = 0, lengths: str = "lognormal",
                    sigma: float = 1.0) -> Graph:
    """Preferential attachment: a star on m+1 vertices, then every new vertex
    links to m distinct earlier vertices drawn with probability proportional
    to degree. |E| = m + (n - m - 1) m."""
    rng = np.random.default_rng(seed)
    us: list[int] = []
    vs: list[int] = []
    repeated: list[int] = []
    for i in range(1, m + 1):  # star centred on 0
        us.append(0)
        vs.append(i)
        repeated.extend([0, i])
    for new in range(m + 1, n):
        targets: set[int] = set()
        while len(targets) < m:
            targets.add(repeated[int(rng.integers(len(repeated)))])
        for t in sorted(targets):
            us.append(t)
            vs.append(new)
            repeated.extend([t, new])
    eu = np.array(us, dtype=np.int64)
    ev = np.array(vs, dtype=np.int64)
    if lengths == "lognormal":
        ell = rng.lognormal(0.0, sigma, size=eu.shape[0])
    elif lengths == "unit":
        ell = np.ones(eu.shape[0])
    else:
        raise ValueError(lengths)
    return Graph(n, eu, ev, ell)


def grid_deleted(nx: int = 300, ny: int = 300, frac: float = 0.15,
                 seed: int = 7) -> Graph:
    """nx x ny grid graph, a fraction `frac` of its edges deleted at random,
    the largest connected component kept (vertices relabelled 0..n-1 in
    increasing original id); lengths U[0.8, 1.2]."""
    rng = np.random.default_rng(seed)
    vid = np.arange(nx * ny, dtype=np.int64).reshape(nx, ny)
    h_u, h_v = vid[:, :-1].ravel(), vid[:, 1:].ravel()
    v_u, v_v = vid[:-1, :].ravel(), vid[1:, :].ravel()
    eu = np.concatenate([h_u, v_u])
    ev = np.concatenate([h_v, v_v])
    n_del = int(round(frac * eu.shape[0]))
    keep = np.ones(eu.shape[0], bool)
    keep[rng.choice(eu.shape[0], size=n_del, replace=False)] = False
    eu, ev = eu[keep], ev[keep]
    comp = _components(nx * ny, eu, ev)
    big = np.bincount(comp).argmax()
    inside = comp == big
    relabel = -np.ones(nx * ny, np.int64)
    relabel[inside] = np.arange(int(inside.sum()))
    ek = inside[eu] & inside[ev]
    eu, ev = relabel[eu[ek]], relabel[ev[ek]]
    lengths = rng.uniform(0.8, 1.2, size=eu.shape[0])
    return Graph(int(inside.sum()), eu, ev, lengths)


def long_edges(n_vertices: int = 200, n_edges: int = 300, n_elems: int = 3072,
               spread: int = 64, h: float = 2.0 ** -9, seed: int = 0) -> Graph:
    """Edges of about n_elems uniform elements each (n_elems +- spread), edge i
    from vertex i mod n_vertices to a uniformly drawn other vertex; length =
    elements x h, so that ceil(length / h) gives the element count back."""
    rng = np.random.default_rng(seed)
    eu = np.arange(n_edges, dtype=np.int64) % n_vertices
    ev = (eu + 1 + rng.integers(n_vertices - 1, size=n_edges)) % n_vertices
    ne = n_elems + rng.integers(-spread, spread, size=n_edges)
    return Graph(n_vertices, eu, ev, ne.astype(np.float64) * h)


def _components(n: int, eu: np.ndarray, ev: np.ndarray) -> np.ndarray:
    parent = np.arange(n)

    def find(a: int) -> int:
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in zip(eu.tolist(), ev.tolist()):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    return np.array([find(i) for i in range(n)])


def random_small_graph(n_vertices: int, n_edges: int, seed: int,
                       lo: float = 0.3, hi: float = 1.5) -> Graph:
    """Random connected multigraph without self-loops: a random spanning tree
    plus extra random edges (parallel edges allowed)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n_vertices)
    us, vs = [], []
    for i in range(1, n_vertices):
        j = int(rng.integers(i))
        us.append(int(perm[j]))
        vs.append(int(perm[i]))
    while len(us) < n_edges:
        a, b = rng.integers(n_vertices, size=2)
        if a != b:
            us.append(int(a))
            vs.append(int(b))
    lengths = rng.uniform(lo, hi, size=len(us))
    return Graph(n_vertices, np.array(us, np.int64), np.array(vs, np.int64), lengths)


def disjoint_union(*graphs: Graph, seed: int = 0) -> Graph:
    """The graphs side by side as one graph with several connected components;
    vertex ids are offset per part and then shuffled by a seeded permutation so
    that the components interleave in the numbering."""
    eu, ev, ln, off = [], [], [], 0
    for g in graphs:
        eu.append(np.asarray(g.edge_u, np.int64) + off)
        ev.append(np.asarray(g.edge_v, np.int64) + off)
        ln.append(np.asarray(g.lengths, np.float64))
        off += g.n_vertices
    perm = np.random.default_rng(seed).permutation(off)
    return Graph(off, perm[np.concatenate(eu)], perm[np.concatenate(ev)], np.concatenate(ln))


@dataclass
class Workload:
    """A named sampling workload: a graph recipe plus the SPDE parameters."""
    name: str
    kappa: float
    beta: float
    k_step: float
    h: float
    n_samples: int
    seed: int
    clip: tuple[int, int] | None = None
    precision: str = "fp64"
    graph_args: dict = field(default_factory=dict)

    def graph(self) -> Graph:
        kind = self.graph_args["kind"]
        args = {k: v for k, v in self.graph_args.items() if k != "kind"}
        return {"square_diagonal": square_diagonal, "rgg": random_geometric,
                "ba": barabasi_albert, "grid": grid_deleted,
                "interval": interval, "long": long_edges}[kind](**args)


WORKLOADS = {
    # 5-edge square with diagonal, FP64, one sample.
    "square5": Workload("square5", kappa=5.0, beta=0.75, k_step=0.5, h=2.0 ** -7,
                        n_samples=1, seed=1, precision="fp64",
                        graph_args={"kind": "square_diagonal", "seed": 0}),
    # Random geometric graph, 2000 vertices, ~5000 edges, mixed precision.
    "rgg2000": Workload("rgg2000", kappa=10.0, beta=0.75, k_step=0.3, h=2.0 ** -10,
                        n_samples=16, seed=1, precision="mixed",
                        graph_args={"kind": "rgg", "n": 2000, "radius": 0.0285,
                                    "seed": 0}),
    # Barabasi-Albert, 20000 vertices, m=3, log-normal lengths, clipped meshes.
    "ba20000": Workload("ba20000", kappa=8.0, beta=0.75, k_step=0.3, h=2.0 ** -9,
                        n_samples=64, seed=1, clip=(2, 4096), precision="mixed",
                        graph_args={"kind": "ba", "n": 20000, "m": 3, "seed": 0}),
    # 300 edges of about 3072 elements (the long edges of ba20000: h = 2^-9,
    # 148 quadrature nodes): the case of the node-parallel sweep profiles.
    "long300": Workload("long300", kappa=8.0, beta=0.75, k_step=0.3, h=2.0 ** -9,
                        n_samples=64, seed=1, precision="mixed",
                        graph_args={"kind": "long", "n_vertices": 200, "n_edges": 300,
                                    "n_elems": 3072, "spread": 64, "h": 2.0 ** -9,
                                    "seed": 0}),
    # 120x120 grid with the 300x300 lattice's parameters and a coarser mesh:
    # more than 4096 vertices and vectors larger than L2 at a few GB on the
    # device (profiles of the vertex PCG).
    "grid120": Workload("grid120", kappa=2.0, beta=0.75, k_step=0.25, h=2.0 ** -6,
                        n_samples=32, seed=1, precision="mixed",
                        graph_args={"kind": "grid", "nx": 120, "ny": 120,
                                    "frac": 0.15, "seed": 7}),
    # 40x40 grid with the 300x300 lattice's parameters and mesh (edges of
    # 410-615 elements, 212 nodes, 32 samples): profiles of its edge kernels.
    "grid40": Workload("grid40", kappa=2.0, beta=0.75, k_step=0.25, h=2.0 ** -9,
                       n_samples=32, seed=1, precision="mixed",
                       graph_args={"kind": "grid", "nx": 40, "ny": 40,
                                   "frac": 0.15, "seed": 7}),
    # 300x300 grid, 15% edges deleted, largest component.
    "grid300": Workload("grid300", kappa=2.0, beta=0.75, k_step=0.25, h=2.0 ** -9,
                        n_samples=32, seed=1, precision="mixed",
                        graph_args={"kind": "grid", "nx": 300, "ny": 300,
                                    "frac": 0.15, "seed": 7}),
}
