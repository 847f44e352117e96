"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: the noise words are bit-exact; FP64 normals agree to a few ulp
(device and host math libraries differ in the last bits); fields agree within a
relative M_L-weighted L2 error of 1e-6 in FP64 mode and 1e-4 in mixed mode
(FP32 edge sweeps). The per-kernel FP64 checks are tighter (1e-9): what is
left there is the PCG tolerance (rtol 1e-12) times the Schur condition number."""
import math

import numpy as np
import pytest

import grf_inputs as gi
from oracle import fem, noise, philox, quadrature, sampler

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

grf = pytest.importorskip("paper_2605_02670_gb300")

TOL = {"fp64": 1e-6, "mixed": 1e-4}


def rel_l2(u, ref, ml):
    u = np.atleast_2d(u)
    ref = np.atleast_2d(ref)
    num = np.sqrt((ml[None, :] * (u - ref) ** 2).sum(axis=1))
    den = np.sqrt((ml[None, :] * ref ** 2).sum(axis=1))
    return float((num / den).max())


def make(g, h=None, n_elems=None, clip=None):
    if n_elems is None and clip is not None:
        n_elems = grf.mesh_elements(g.lengths, h, clip)
    G = grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=h, n_elems=n_elems)
    m = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=h, n_elems=n_elems,
                       clip=None)
    return G, m


GRAPHS = {
    "square5": lambda: (gi.square_diagonal(0), 2.0 ** -7),
    "interval": lambda: (gi.interval(1.3), 0.05),
    "random12": lambda: (gi.random_small_graph(12, 20, 3), 0.07),
    "short_edges": lambda: (gi.Graph(5, np.array([0, 1, 2, 3, 0, 1]), np.array([1, 2, 3, 4, 2, 0]),
                                     np.array([0.05, 0.11, 0.2, 0.9, 0.15, 0.33])), 0.1),
    "isolated": lambda: (gi.Graph(6, np.array([0, 2, 2]), np.array([2, 4, 5]),
                                  np.array([0.7, 1.2, 0.4])), 0.03),
}


# ---------------------------------------------------------------- noise


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("seed", [1, 0xDEADBEEF12345678])
def test_noise_words_bit_exact(name, seed):
    g, h = GRAPHS[name]()
    G, m = make(g, h)
    words = G.noise(seed, 5, raw=True).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(words, philox.noise_words(seed, m.n_dofs, 5))


def test_noise_words_match_curand_philox(tmp_path):
    """The noise words against a second Philox4x32-10: cuRAND's device
    generator (run through a small test-only kernel, tests/curand_philox_words.cu)
    started at the same key (seed) and counter (block q, sample s). Both follow
    the published Random123 definition; this pins the key and counter layout
    on the GPU independently of the oracle."""
    import ctypes
    import subprocess
    from pathlib import Path

    from paper_2605_02670_gb300 import build as grf_build

    src = Path(__file__).with_name("curand_philox_words.cu")
    lib = tmp_path / "libcurand_blocks.so"
    subprocess.run([grf_build.nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                    "-shared", "-Xcompiler", "-fPIC", "-o", str(lib), str(src)], check=True)
    cl = ctypes.CDLL(str(lib))
    cl.curand_philox_blocks.restype = ctypes.c_int
    cl.curand_philox_blocks.argtypes = [ctypes.c_ulonglong, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p]
    g, h = GRAPHS["square5"]()
    G, m = make(g, h)
    S = 7
    nq = m.n_dofs // 4  # whole blocks only
    for seed in (1, 0xDEADBEEF12345678):
        words = G.noise(seed, S, raw=True).cpu().numpy().view(np.uint32)
        s_idx = np.repeat(np.arange(S, dtype=np.int32), nq)
        q_idx = np.tile(np.arange(nq, dtype=np.int64), S)
        d_s = torch.from_numpy(s_idx).cuda()
        d_q = torch.from_numpy(q_idx).cuda()
        d_out = torch.empty((s_idx.size, 4), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        rc = cl.curand_philox_blocks(seed, d_s.data_ptr(), d_q.data_ptr(), s_idx.size,
                                     d_out.data_ptr())
        assert rc == 0
        ref = d_out.cpu().numpy().view(np.uint32).reshape(S, nq * 4)
        np.testing.assert_array_equal(words[:, :nq * 4], ref)


@pytest.mark.parametrize("name", ["square5", "random12", "isolated"])
def test_noise_values(name):
    g, h = GRAPHS[name]()
    G, m = make(g, h)
    b = G.noise(7, 6).cpu().numpy()
    ref = noise.white_noise(fem.lumped_mass(m), 7, 6)
    np.testing.assert_allclose(b, ref, rtol=1e-13, atol=1e-14)


def test_noise_large_counter_range():
    # more than 2^32 / 4 ... only the counter split matters; use a large DOF count
    g = gi.Graph(2, np.array([0]), np.array([1]), np.array([1.0]))
    G, m = make(g, n_elems=[3_000_001])
    words = G.noise(3, 2, raw=True).cpu().numpy().view(np.uint32)
    ref = philox.noise_words(3, m.n_dofs, 2)
    np.testing.assert_array_equal(words[:, -1000:], ref[:, -1000:])
    np.testing.assert_array_equal(words[:, :1000], ref[:, :1000])


# ---------------------------------------------------------------- Schur blocks


@pytest.mark.parametrize("name", ["square5", "random12", "short_edges", "isolated"])
@pytest.mark.parametrize("alpha,gamma", [(1.0, 1e-25), (1.0, 1e-3), (1.0, 0.7), (1.0, 4e9),
                                         (0.0, 1.0)])
def test_schur_blocks(name, alpha, gamma):
    g, h = GRAPHS[name]()
    G, m = make(g, h)
    kappa = 2.3
    diag, off = G.schur(kappa, alpha, gamma)
    ml, _, kmat = sampler.assemble(m, kappa)
    s = sampler.vertex_schur_dense(m, ml, kmat, gamma, alpha=alpha)
    np.testing.assert_allclose(diag.cpu().numpy(), np.diag(s), rtol=1e-11)
    # off-diagonal: the oracle's S_uv sums over parallel edges
    offs = off.cpu().numpy()
    dense = np.zeros_like(s)
    for e in range(g.n_edges):
        a, b = m.edge_u[e], m.edge_v[e]
        dense[a, b] += offs[e]
        dense[b, a] += offs[e]
    mask = ~np.eye(s.shape[0], dtype=bool)
    np.testing.assert_allclose(dense[mask], s[mask], rtol=1e-10,
                               atol=1e-13 * np.abs(np.diag(s)).max())


# ---------------------------------------------------------------- condensation + PCG


@pytest.mark.parametrize("precision,interior", [("fp64", "auto"), ("mixed", "thomas"),
                                                ("mixed", "spectral")])
@pytest.mark.parametrize("gamma", [1e-12, 0.05, 3.0, 1e7])
def test_vertex_condensation_and_pcg(precision, interior, gamma):
    g, h = GRAPHS["random12"]()
    G, m = make(g, h)
    kappa = 1.7
    ml, _, kmat = sampler.assemble(m, kappa)
    rhs = noise.white_noise(ml, 4, 5)
    gv, uv, st = G.vertex_solve(kappa, 1.0, gamma, torch.tensor(rhs, device="cuda"),
                                precision=precision, interior=interior)
    g_ref, u_ref = sampler.vertex_condensation(m, ml, kmat, gamma, rhs)
    tol = 1e-10 if precision == "fp64" else 1e-5
    for got, ref in ((gv, g_ref), (uv, u_ref)):
        got = got.cpu().numpy()
        err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() < tol, err
    assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0


# ---------------------------------------------------------------- general right-hand side


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(GRAPHS))
def test_apply_matches_oracle(precision, name):
    g, h = GRAPHS[name]()
    G, m = make(g, h)
    kappa = 3.1
    ml, _, kmat = sampler.assemble(m, kappa)
    rng = np.random.default_rng(5)
    rhs = rng.standard_normal((3, m.n_dofs))
    t = np.array([1e-9, 0.01, 1.0, 30.0, 1e6])
    w = np.array([0.3, 1.0, 2.0, 0.5, 1e-3])
    alpha = np.ones_like(t)
    out, st = G.apply(kappa, alpha, t, w, torch.tensor(rhs, device="cuda"), precision=precision,
                      out_dtype="f64")
    ref = sampler.shifted_sum(ml, kmat, rhs, t, w)
    assert rel_l2(out.cpu().numpy(), ref, ml) < TOL[precision] / 10
    # the stiffness node (alpha = 0) used for the integer part of beta
    out0, _ = G.apply(kappa, [0.0], [1.0], [1.0], torch.tensor(rhs, device="cuda"),
                      precision=precision, out_dtype="f64")
    ref0 = sampler.stiff_solve(kmat, rhs)
    assert rel_l2(out0.cpu().numpy(), ref0, ml) < TOL[precision] / 10


# ---------------------------------------------------------------- whole sampler


@pytest.mark.parametrize("precision,interior", [("fp64", "auto"), ("mixed", "thomas"),
                                                ("mixed", "spectral"), ("mixed", "spectral_tc"),
                                                ("mixed", "spectral_umma")])
@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("beta", [0.3, 0.75])
def test_sample_matches_oracle(precision, interior, name, beta):
    g, h = GRAPHS[name]()
    G, m = make(g, h)
    kappa, k, seed, S = 4.0, 0.45, 11, 5
    u, st = G.sample(kappa, beta, k, seed, S, precision=precision, out_dtype="f64",
                     interior=interior)
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, h=h)
    ml = fem.lumped_mass(m)
    assert rel_l2(u.cpu().numpy(), ref, ml) < TOL[precision]
    km, kp = quadrature.limits(beta, k)
    assert st["n_nodes"] == km + kp + 1 and st["n_systems"] == (km + kp + 1) * S
    assert st["n_unconverged"] == 0


@pytest.mark.parametrize("layout", ["per_system", "staged", "staged_pairs"])
@pytest.mark.parametrize("name", ["square5", "random12", "isolated"])
def test_sample_pcg_layouts(layout, name):
    g, h = GRAPHS[name]()
    G, m = make(g, h)
    kappa, beta, k, seed, S = 4.0, 0.6, 0.45, 13, 7
    u, st = G.sample(kappa, beta, k, seed, S, precision="mixed", out_dtype="f64",
                     pcg_layout=layout)
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, h=h)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < TOL["mixed"]
    assert st["n_unconverged"] == 0


@pytest.mark.parametrize("layout", ["staged", "staged_pairs"])
@pytest.mark.parametrize("nx", [12, 20, 30, 40, 50])
def test_sample_group_pcg_every_vertex_split(nx, layout):
    """The sample-group PCG layouts on grids of about 144, 400, 870, 1550 and
    2400 kept vertices: every vertices-per-thread split of the 512-thread
    groups of 4 samples and of the 256-thread pairs, with a ragged last sample
    group (S = 5)."""
    g = gi.grid_deleted(nx, nx, 0.15, 2)
    G, m = make(g, 0.5)
    kappa, beta, k, seed, S = 1.5, 0.7, 0.5, 17, 5
    u, st = G.sample(kappa, beta, k, seed, S, precision="mixed", out_dtype="f64",
                     pcg_layout=layout)
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, h=0.5)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < TOL["mixed"]
    assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0
    u1, s1 = G.sample(kappa, beta, k, seed, S, precision="mixed", out_dtype="f64",
                      pcg_layout="per_system")
    assert rel_l2(u.cpu().numpy(), u1.cpu().numpy(), fem.lumped_mass(m)) < TOL["mixed"] / 10


@pytest.mark.parametrize("layout", ["staged", "staged_pairs", "per_system"])
@pytest.mark.parametrize("parts", [(12, 30, 60), (20, 40, 300)])
def test_sample_pcg_disconnected_multigraph(layout, parts):
    """Several connected components whose vertex ids interleave, with parallel
    edges, in the sample-group layouts (which renumber the vertices component by
    component) and one CTA per system: 236 and 742 kept vertices."""
    nx, n_small, n_rand = parts
    g = gi.disjoint_union(gi.grid_deleted(nx, nx, 0.15, 3),
                          gi.random_small_graph(n_rand, 2 * n_rand, 4),
                          gi.random_small_graph(n_small, n_small + 6, 5),
                          gi.interval(0.8), seed=nx)
    G, m = make(g, 0.2)
    kappa, beta, k, seed, S = 2.0, 0.65, 0.5, 23, 6
    u, st = G.sample(kappa, beta, k, seed, S, precision="mixed", out_dtype="f64",
                     pcg_layout=layout)
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, h=0.2)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < TOL["mixed"]
    assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sample_large_graph_global_vectors(precision):
    """About 9 000 kept vertices: the per-system PCG keeps its vectors in global
    memory (they do not fit shared memory), in both precisions; the group layout
    falls back to it too."""
    g = gi.grid_deleted(105, 105, 0.15, 4)
    G, m = make(g, 0.45)
    assert G.n_kept > 8600
    kappa, beta, k, seed, S = 1.5, 0.7, 0.5, 19, 3
    u, st = G.sample(kappa, beta, k, seed, S, precision=precision, out_dtype="f64",
                     pcg_layout="per_system")
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, h=0.45)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < TOL[precision]
    assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sample_large_disconnected_graph_global_vectors(precision):
    """10 554 kept vertices in three components with interleaved ids (two grids
    with deleted edges and a small multigraph with parallel edges): the
    per-system PCG with its vectors in global memory, which in mixed precision
    keeps them in vertex order (the group layouts renumber, this one does not)."""
    g = gi.disjoint_union(gi.grid_deleted(75, 75, 0.15, 6), gi.grid_deleted(70, 70, 0.15, 7),
                          gi.random_small_graph(40, 50, 9), seed=5)
    G, m = make(g, 0.45)
    assert G.n_kept > 10000
    kappa, beta, k, seed, S = 1.5, 0.7, 0.5, 19, 3
    u, st = G.sample(kappa, beta, k, seed, S, precision=precision, out_dtype="f64",
                     pcg_layout="per_system")
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, h=0.45)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < TOL[precision]
    assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0


@pytest.mark.parametrize("precision,sg,interior", [
    ("fp64", 0, "thomas"), ("mixed", 1, "thomas"), ("mixed", 2, "thomas"), ("mixed", 4, "thomas"),
    ("mixed", 1, "spectral"), ("mixed", 4, "spectral"), ("mixed", 4, "spectral_tc"),
    ("mixed", 4, "spectral_umma")])
def test_sample_every_recovery_bin(precision, sg, interior):
    """Edge interiors from 1 to 4999 nodes: every register-resident bin of the
    Thomas recovery (one warp with 1, 2, 4, 8 nodes per lane; 2 to 16 warps),
    each samples-per-lane variant, the sequential kernel for edges longer than
    the largest bin, and every bin of the spectral path (m <= 64, 128, 256,
    384, 512, 768, 1024) with the longer edges left to Thomas."""
    ne = [2, 33, 65, 129, 257, 513, 1025, 2049, 4097, 5000, 3, 31, 301, 701]
    E = len(ne)
    eu = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 0, 3, 1, 2])
    ev = np.array([1, 2, 3, 4, 5, 6, 7, 8, 9, 0, 5, 8, 6, 9])
    lengths = np.array(ne) * 1e-3 * np.linspace(0.8, 1.2, E)
    g = gi.Graph(10, eu, ev, lengths)
    G, m = make(g, n_elems=ne)
    kappa, beta, k, seed, S = 6.0, 0.6, 0.5, 21, 6
    u, st = G.sample(kappa, beta, k, seed, S, precision=precision, out_dtype="f64",
                     recover_sg=sg, interior=interior)
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, n_elems=ne)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < TOL[precision]


@pytest.mark.parametrize("sweep,interior", [("nodes", "thomas"), ("segments", "thomas"),
                                            ("nodes", "spectral")])
@pytest.mark.parametrize("S", [6, 8])
@pytest.mark.parametrize("h", [1e-3, 2e-2])
def test_sample_node_sweeps(sweep, interior, S, h):
    """The node-parallel FP32 sweeps (one warp per edge and 4 samples, twisted
    factorisation in the recovery) against the oracle: interiors of 1 to 2999
    nodes, so that the 8-node output blocks end ragged and the two end zones of
    unconverged pivots overlap (small h: j theta < 9 along whole edges) or
    leave a long converged middle (large h); S = 6 leaves a group of 2 samples
    (scalar row loads), S = 8 full groups (vector loads)."""
    ne = [2, 3, 4, 8, 9, 10, 16, 17, 18, 300, 1025, 3000]
    E = len(ne)
    eu = np.array([0, 1, 2, 3, 4, 5, 6, 7, 0, 2, 4, 6])
    ev = np.array([1, 2, 3, 4, 5, 6, 7, 0, 4, 6, 1, 3])
    lengths = np.array(ne) * h
    g = gi.Graph(8, eu, ev, lengths)
    G, m = make(g, n_elems=ne)
    kappa, beta, k, seed = 6.0, 0.6, 0.5, 23
    u, st = G.sample(kappa, beta, k, seed, S, precision="mixed", out_dtype="f64",
                     interior=interior, sweep=sweep)
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, n_elems=ne)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < TOL["mixed"]
    assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0


@pytest.mark.parametrize("beta", [0.25, 0.75])
def test_node_sweeps_many_nodes_per_lane(beta):
    """k = 0.3 gives 148 quadrature nodes at beta = 0.25 and 0.75: five nodes per
    lane; the node and segment sweeps agree, and both match the oracle."""
    ne = [40, 600, 1500]
    g = gi.Graph(3, np.array([0, 1, 2]), np.array([1, 2, 0]), np.array(ne) * 2.0 ** -9)
    G, m = make(g, n_elems=ne)
    kappa, k, seed, S = 8.0, 0.3, 5, 4
    un, _ = G.sample(kappa, beta, k, seed, S, precision="mixed", out_dtype="f64",
                     interior="thomas", sweep="nodes")
    us, _ = G.sample(kappa, beta, k, seed, S, precision="mixed", out_dtype="f64",
                     interior="thomas", sweep="segments")
    ml = fem.lumped_mass(m)
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, n_elems=ne)
    assert rel_l2(un.cpu().numpy(), ref, ml) < TOL["mixed"]
    assert rel_l2(us.cpu().numpy(), ref, ml) < TOL["mixed"]
    assert rel_l2(un.cpu().numpy(), us.cpu().numpy(), ml) < TOL["mixed"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("beta", [1.0, 1.25, 2.0, 2.6])
def test_sample_integer_powers(precision, beta):
    g, h = GRAPHS["square5"]()
    G, m = make(g, 2.0 ** -5)
    kappa, k, seed, S = 2.0, 0.5, 3, 2
    u, st = G.sample(kappa, beta, k, seed, S, precision=precision, out_dtype="f64")
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, h=2.0 ** -5)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < TOL[precision]


def test_sample_square5_workload_fp64_and_f32_output():
    w = gi.WORKLOADS["square5"]
    g = w.graph()
    G, m = make(g, w.h)
    _, ref, _ = sampler.sample(g, w.kappa, w.beta, w.k_step, w.seed, 1, h=w.h)
    ml = fem.lumped_mass(m)
    u, _ = G.sample(w.kappa, w.beta, w.k_step, w.seed, 1, precision="fp64")
    assert rel_l2(u.cpu().numpy(), ref, ml) < 1e-6
    u32, _ = G.sample(w.kappa, w.beta, w.k_step, w.seed, 1, precision="fp64", out_dtype="f32")
    assert u32.dtype == torch.float32
    assert rel_l2(u32.double().cpu().numpy(), ref, ml) < 1e-6
    uh, _ = G.sample_host(w.kappa, w.beta, w.k_step, w.seed, 1, precision="fp64")
    np.testing.assert_array_equal(uh, u.cpu().numpy())


def test_sample_is_deterministic_in_seed_and_sample_index():
    g, h = GRAPHS["random12"]()
    G, _ = make(g, h)
    a, _ = G.sample(2.0, 0.6, 0.5, 99, 6, precision="mixed")
    b, _ = G.sample(2.0, 0.6, 0.5, 99, 3, precision="mixed")
    # sample s depends only on (seed, s): the first three rows agree
    np.testing.assert_allclose(a[:3].cpu().numpy(), b.cpu().numpy(), rtol=1e-5, atol=1e-7)
    c, _ = G.sample(2.0, 0.6, 0.5, 100, 3, precision="mixed")
    assert not np.allclose(c.cpu().numpy(), b.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cuda_graph_replay_matches_direct_calls(precision):
    g, h = GRAPHS["random12"]()
    G, m = make(g, h)
    ml = fem.lumped_mass(m)
    tol = 1e-12 if precision == "fp64" else 1e-6
    out = torch.empty((5, G.n_dofs), dtype=torch.float64, device="cuda")
    for beta, seed in [(0.6, 3), (0.6, 4), (1.3, 4), (0.6, 3)]:
        direct, st_d = G.sample(2.5, beta, 0.45, seed, 5, precision=precision, out_dtype="f64")
        graphed, st_g = G.sample(2.5, beta, 0.45, seed, 5, precision=precision, out_dtype="f64",
                                 out=out, use_graph=True)
        assert rel_l2(graphed.cpu().numpy(), direct.cpu().numpy(), ml) < tol
        assert st_g["n_nodes"] == st_d["n_nodes"] and st_g["n_systems"] == st_d["n_systems"]
        assert st_g["pcg_iters_total"] > 0
        # and the replay really used this seed: matches the oracle
        _, ref, _ = sampler.sample(g, 2.5, beta, 0.45, seed, 5, h=h)
        assert rel_l2(graphed.cpu().numpy(), ref, ml) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_reports_phase_times(precision):
    """With phase timing a replayed graph records the phase events as event
    record nodes: every replay reports its own device time per phase, and the
    field agrees with the untimed replay's."""
    g, h = GRAPHS["random12"]()
    G, m = make(g, h)
    ml = fem.lumped_mass(m)
    tol = 1e-12 if precision == "fp64" else 1e-6
    out = torch.empty((4, G.n_dofs), dtype=torch.float64, device="cuda")
    plain = {}
    for seed in (8, 9):
        u, _ = G.sample(2.5, 0.6, 0.45, seed, 4, precision=precision, out_dtype="f64", out=out,
                        use_graph=True)
        plain[seed] = u.cpu().numpy()
    for seed in (8, 9):  # the timed graph: captured, then replayed
        u, st = G.sample(2.5, 0.6, 0.45, seed, 4, precision=precision, out_dtype="f64", out=out,
                         use_graph=True, timing=True)
        assert rel_l2(u.cpu().numpy(), plain[seed], ml) < tol
        ph = st["phase_ms"]
        for k in ("noise", "schur", "condense", "pcg", "recover"):
            assert 0.0 < ph[k] < 1e3, (k, ph)
        assert ph["precond_net"] == 0.0
    for seed in (8, 9):  # only the PCG phase timed: its two events alone
        u, st = G.sample(2.5, 0.6, 0.45, seed, 4, precision=precision, out_dtype="f64", out=out,
                         use_graph=True, timing=["pcg"])
        assert rel_l2(u.cpu().numpy(), plain[seed], ml) < tol
        ph = st["phase_ms"]
        assert 0.0 < ph["pcg"] < 1e3
        assert all(v == 0.0 for k, v in ph.items() if k != "pcg"), ph


def test_sample_host_graph_replay_across_calls():
    """grf_sample_host keeps its device output on the handle, so a captured
    graph is replayed (not re-captured) by later calls and still follows the
    seed; a larger sample count regrows the buffer and re-captures."""
    g, h = GRAPHS["random12"]()
    G, m = make(g, h)
    ml = fem.lumped_mass(m)
    for seed, S in ((5, 3), (6, 3), (7, 5), (5, 3)):
        d, _ = G.sample_host(2.0, 0.6, 0.5, seed, S, precision="mixed", out_dtype="f64")
        r, st = G.sample_host(2.0, 0.6, 0.5, seed, S, precision="mixed", out_dtype="f64",
                              use_graph=True)
        assert rel_l2(r, d, ml) < 1e-6 and st["n_unconverged"] == 0


def test_autotune_returns_working_knobs():
    g, h = GRAPHS["random12"]()
    G, m = make(g, h)
    knobs, ms = G.autotune(3.0, 0.7, 0.5, 8, precision="mixed")
    assert knobs["pcg_layout"] in ("per_system", "staged", "staged_pairs")
    assert knobs["recover_sg"] in (1, 2, 4)
    assert knobs["interior"] in ("thomas", "spectral", "spectral_tc")
    assert knobs["sweep"] in ("auto", "segments", "nodes")
    assert ms > 0
    u, _ = G.sample(3.0, 0.7, 0.5, 9, 8, precision="mixed", out_dtype="f64", **knobs)
    _, ref, _ = sampler.sample(g, 3.0, 0.7, 0.5, 9, 8, h=h)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < TOL["mixed"]


def test_zero_samples_and_max_iter_flag():
    g, h = GRAPHS["random12"]()
    G, _ = make(g, h)
    out, st = G.sample(2.0, 0.6, 0.5, 1, 0)
    assert out.shape == (0, G.n_dofs) and st["n_systems"] == 0
    with pytest.raises(grf.GrfError) as ei:
        G.sample(0.3, 0.6, 0.5, 1, 2, max_iter=1, rtol=1e-14)
    assert ei.value.code == grf.GRF_ENOCONV
    u, st = G.sample(0.3, 0.6, 0.5, 1, 2, max_iter=1, rtol=1e-14, allow_noconv=True)
    assert st["n_unconverged"] > 0 and np.isfinite(u.cpu().numpy()).all()


# ---------------------------------------------------------------- bench-size workloads


def _sampled_node_check(wname, nodes_t, S, precision):
    """Full-size graph, bench launch configuration, single shifted nodes:
    the oracle factorises one node at a time."""
    w = gi.WORKLOADS[wname]
    g = w.graph()
    ne = grf.mesh_elements(g.lengths, w.h, w.clip)
    G, m = make(g, n_elems=ne)
    ml, _, kmat = sampler.assemble(m, w.kappa)
    b = noise.white_noise(ml, w.seed, S)
    bt = torch.tensor(b, device="cuda")
    for t in nodes_t:
        out, _ = G.apply(w.kappa, [1.0], [t], [1.0], bt, precision=precision, out_dtype="f64")
        ref = sampler.shifted_sum(ml, kmat, b, [t], [1.0])
        assert rel_l2(out.cpu().numpy(), ref, ml) < TOL[precision], t


def test_rgg2000_full_size_sampled_nodes():
    w = gi.WORKLOADS["rgg2000"]
    t, _ = quadrature.nodes(w.beta, w.k_step)
    _sampled_node_check("rgg2000", [t[0], t[len(t) // 2], t[-1]], 4, "mixed")


# ---------------------------------------------------------------- preconditioners


@pytest.mark.parametrize("precision,layout", [("fp64", "per_system"), ("mixed", "per_system"),
                                              ("mixed", "staged")])
@pytest.mark.parametrize("name", ["random12", "square5", "isolated"])
def test_neumann_neumann_preconditioner_matches_oracle(precision, layout, name):
    """The paper's Neumann-Neumann preconditioner changes how PCG converges,
    not what it converges to: same field tolerance as Jacobi."""
    g, h = GRAPHS[name]()
    G, m = make(g, h)
    kappa, beta, k, seed, S = 3.0, 0.7, 0.45, 19, 6
    u, st = G.sample(kappa, beta, k, seed, S, precision=precision, out_dtype="f64",
                     pcg_layout=layout, precond="neumann")
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, h=h)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < TOL[precision]
    assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0
    assert st["n_precond_fallback"] == 0


@pytest.mark.parametrize("layout", ["per_system", "staged"])
def test_neumann_neumann_on_larger_grid(layout):
    g = gi.grid_deleted(40, 40, 0.15, 2)
    G, m = make(g, 0.5)
    kappa, beta, k, seed, S = 1.5, 0.7, 0.5, 23, 5
    u, st = G.sample(kappa, beta, k, seed, S, precision="mixed", out_dtype="f64",
                     pcg_layout=layout, precond="neumann")
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, h=0.5)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < TOL["mixed"]
    assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0


def test_neumann_neumann_vertex_solve():
    g, h = GRAPHS["random12"]()
    G, m = make(g, h)
    kappa = 1.7
    ml, _, kmat = sampler.assemble(m, kappa)
    rhs = noise.white_noise(ml, 4, 5)
    for precision, tol in (("fp64", 1e-10), ("mixed", 1e-5)):
        gv, uv, st = G.vertex_solve(kappa, 1.0, 0.05, torch.tensor(rhs, device="cuda"),
                                    precision=precision, precond="neumann")
        _, u_ref = sampler.vertex_condensation(m, ml, kmat, 0.05, rhs)
        err = np.linalg.norm(uv.cpu().numpy() - u_ref, axis=1) / np.linalg.norm(u_ref, axis=1)
        assert err.max() < tol, (precision, err)


def test_sample_host_stream_equals_separate_host_calls():
    g = gi.random_small_graph(12, 20, 3)
    G = grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=0.05)
    kw = dict(precision="mixed", out_dtype="f32", use_graph=True, interior="spectral_umma")
    seeds = [5, 6, 7]
    outs, st = G.sample_host_stream(2.0, 0.7, 0.4, seeds, 4, **kw)
    assert st["n_unconverged"] == 0 and st["pcg_iters_total"] > 0
    for sd, o in zip(seeds, outs):
        ref, _ = G.sample_host(2.0, 0.7, 0.4, sd, 4, **kw)
        np.testing.assert_array_equal(o, ref)
    # one buffer reused for every call holds the last call's field
    buf = np.empty_like(outs[0])
    G.sample_host_stream(2.0, 0.7, 0.4, seeds, 4, outs=[buf, buf, buf], **kw)
    np.testing.assert_array_equal(buf, outs[-1])


@pytest.mark.parametrize("interior", ["thomas", "spectral", "spectral_umma"])
def test_apply_extreme_shifts_mixed(interior):
    """Shifts far outside the FP32 range (the outer sinc nodes of small steps
    reach t = e^133): the nodes are rescaled to O(1) before the FP32 kernels."""
    g = gi.random_small_graph(12, 20, 3)
    G = grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=0.01)
    m = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=0.01)
    kappa = 1.3
    ml, _, kmat = sampler.assemble(m, kappa)
    rhs = np.random.default_rng(8).standard_normal((3, m.n_dofs))
    t = np.array([1e-32, 1e-12, 1.0, 1e25, 1e45, 6e57])
    w = np.array([1e-22, 1e-6, 1.0, 1e15, 1e34, 3e43])
    out, st = G.apply(kappa, np.ones_like(t), t, w, torch.tensor(rhs, device="cuda"),
                      precision="mixed", out_dtype="f64", interior=interior)
    assert st["numeric_flag"] == 0 and st["n_unconverged"] == 0
    ref = sampler.shifted_sum(ml, kmat, rhs, t, w)
    num = np.sqrt((ml[None, :] * (out.cpu().numpy() - ref) ** 2).sum(axis=1))
    den = np.sqrt((ml[None, :] * ref ** 2).sum(axis=1))
    assert (num / den).max() < 1e-5


def test_apply_shift_below_the_fp32_range_is_refused_in_mixed():
    """t = 1e-45 on h = 0.01 gives c = t / h = 1e-43 (subnormal in FP32): the
    mixed path refuses the node, FP64 computes it."""
    g = gi.random_small_graph(12, 20, 3)
    G = grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=0.01)
    m = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=0.01)
    kappa = 1.3
    ml, _, kmat = sampler.assemble(m, kappa)
    rhs = np.random.default_rng(8).standard_normal((2, m.n_dofs))
    t, w = np.array([1e-45, 1.0]), np.array([1e-30, 1.0])
    with pytest.raises(grf.GrfError) as ei:
        G.apply(kappa, np.ones_like(t), t, w, torch.tensor(rhs, device="cuda"),
                precision="mixed", out_dtype="f64")
    assert ei.value.code == grf.GRF_ENOTSUP
    out, _ = G.apply(kappa, np.ones_like(t), t, w, torch.tensor(rhs, device="cuda"),
                     precision="fp64")
    ref = sampler.shifted_sum(ml, kmat, rhs, t, w)
    num = np.sqrt((ml[None, :] * (out.cpu().numpy() - ref) ** 2).sum(axis=1))
    den = np.sqrt((ml[None, :] * ref ** 2).sum(axis=1))
    assert (num / den).max() < 1e-6
