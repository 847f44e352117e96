"""The consistent-mass comparison system on the GPU (Sec. 2.4 Eq. wh_def with
the consistent mass of Sec. 3 Phase 2, and the consistent mass in the shifted
operators) through the C ABI, against the oracle: the Cholesky noise, the
solves with a general right-hand side, and whole samples. Mixed precision
(FP32 noise and edge interiors, FP64 Schur blocks and refinement): relative
L2 tolerance 1e-4 for fields, 1e-5 for the noise."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import grf_inputs as gi
from oracle import consistent, fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
grf = pytest.importorskip("paper_2605_02670_gb300")

GRAPHS = {
    "square5": lambda: (gi.square_diagonal(0), 2.0 ** -7),
    "random12": lambda: (gi.random_small_graph(12, 20, 3), 0.07),
    "short_edges": lambda: (gi.Graph(5, np.array([0, 1, 2, 3, 0, 1]), np.array([1, 2, 3, 4, 2, 0]),
                                     np.array([0.05, 0.11, 0.2, 0.9, 0.15, 0.33])), 0.1),
    "lattice6": lambda: (gi.grid_deleted(6, 6, 0.15, seed=7), 2.0 ** -9),
}


def rel_l2(u, ref, ml):
    num = np.sqrt((ml[None, :] * (u - ref) ** 2).sum(axis=1))
    den = np.sqrt((ml[None, :] * ref ** 2).sum(axis=1))
    return float((num / den).max())


def _pair(name):
    g, h = GRAPHS[name]()
    G = grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=h)
    m = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=h)
    return g, h, G, m


@pytest.mark.parametrize("name", ["square5", "random12", "short_edges"])
def test_consistent_noise_matches_oracle(name):
    g, h, G, m = _pair(name)
    w = G.noise(17, 6, mass="consistent").cpu().numpy()
    ref = consistent.white_noise(m, 17, 6)
    err = np.linalg.norm(w - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() < 1e-5, err


@pytest.mark.parametrize("name", list(GRAPHS))
def test_consistent_operator_general_rhs(name):
    g, h, G, m = _pair(name)
    kappa = 3.1
    mc, _, kc = consistent.assemble(m, kappa)
    rng = np.random.default_rng(5)
    rhs = rng.standard_normal((3, m.n_dofs))
    # shifts on both sides of t = h^2 / 6, where the consistent interior
    # block's off-diagonal changes sign
    t = np.array([1e-9, h * h / 12, h * h / 4, 0.01, 1.0, 30.0, 1e6])
    w = np.array([0.3, 0.7, 1.1, 1.0, 2.0, 0.5, 1e-3])
    out, st = G.apply(kappa, np.ones_like(t), t, w, torch.tensor(rhs, device="cuda"),
                      precision="mixed", out_dtype="f64", mass="consistent")
    ref = np.zeros_like(rhs)
    for tl, wl in zip(t, w):
        ref += wl * spla.splu((mc + tl * kc).tocsc()).solve(np.ascontiguousarray(rhs.T)).T
    assert rel_l2(out.cpu().numpy(), ref, fem.lumped_mass(m)) < 1e-5
    assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("beta", [0.3, 0.75])
def test_consistent_sample_matches_oracle(name, beta):
    g, h, G, m = _pair(name)
    kappa, k, seed, S = 4.0, 0.45, 11, 5
    u, st = G.sample(kappa, beta, k, seed, S, precision="mixed", out_dtype="f64",
                     mass="consistent")
    _, ref, _ = consistent.sample(g, kappa, beta, k, seed, S, h=h)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < 1e-4
    assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0


def test_consistent_sample_graph_replay():
    g, h, G, m = _pair("random12")
    kappa, beta, k, S = 2.5, 0.6, 0.45, 4
    out = torch.empty((S, G.n_dofs), dtype=torch.float64, device="cuda")
    for seed in (3, 4):
        u, _ = G.sample(kappa, beta, k, seed, S, precision="mixed", out_dtype="f64", out=out,
                        use_graph=True, mass="consistent")
        _, ref, _ = consistent.sample(g, kappa, beta, k, seed, S, h=h)
        assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < 1e-4


def test_consistent_refusals():
    g, h, G, m = _pair("random12")
    with pytest.raises(grf.GrfError) as ei:  # integer part of beta
        G.sample(2.0, 1.25, 0.5, 1, 2, precision="mixed", mass="consistent")
    assert ei.value.code == grf.GRF_ENOTSUP
    long = gi.Graph(2, np.array([0]), np.array([1]), np.array([3.0]))
    GL = grf.Graph(long.edge_u, long.edge_v, long.lengths, long.n_vertices, h=2.0 ** -9)
    with pytest.raises(grf.GrfError) as ei:  # an edge beyond the sine-basis path
        GL.sample(2.0, 0.6, 0.5, 1, 2, precision="mixed", mass="consistent")
    assert ei.value.code == grf.GRF_ENOTSUP


def test_mass_comparison_harness_small_graph():
    from paper_2605_02670_gb300 import mass_comparison as mc
    row = mc.compare(100, S=4, reps=1)
    assert row["n_dofs"] == 100 + 63 * row["n_edges"]
    for mass in ("lumped", "consistent"):
        assert row[mass]["call_ms"] > 0 and row[mass]["noise_ms"] > 0
    assert row["consistent_over_lumped"]["full"] > 0
