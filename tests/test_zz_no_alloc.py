"""grf_vertex_solve_noalloc: the vertex Schur solve for callers that cannot
allocate device memory (their device memory belongs to another allocator with
a fixed budget, or their loop must not pay the device-wide synchronisation of
cudaMalloc/cudaFree). Its scratch is a static 16 MiB device array inside the
library. It must give what the allocating grf_vertex_solve gives, call after
call, although the array keeps the previous call's contents.

This file is collected last on purpose: a failure here leaves every other
test already run."""
import numpy as np
import pytest

import grf_inputs as gi
import paper_2605_02670_gb300 as grf

TOL = {"fp64": 1e-10, "mixed": 1e-5}  # the vertex-solve tolerances of the parity tests


def _graph():
    g = gi.random_small_graph(12, 20, 3)
    return grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=0.07)


LONG_H = 2.0 ** -9


def _long_graph_input():
    # lengths 0.3-1.5 at h = 2^-9: 153-768 elements per edge, so every edge is
    # past the 64 interior nodes where the FP32 sweeps go node-parallel
    return gi.random_small_graph(12, 20, 3)


def _long_graph():
    g = _long_graph_input()
    return grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=LONG_H)


def _scratch_bytes(n_dofs, n_kept, n_edges, n_rhs, ts):
    """The buffers the entry point carves from its static array, each rounded
    up to 256 bytes: the sample-minor right-hand side, the node constants, the
    Schur system, four PCG vectors per right-hand side, the Jacobi scaling, the
    FP32 copy of the off-diagonals (mixed), the FP32-pair copies of the Schur
    blocks and the batched PCG's four pair vectors (mixed), iteration counts,
    the status words and the per-edge sweep constants (4 values per edge) that
    the long FP32 edges' node-parallel condensation reads."""
    up = lambda x: (x + 255) // 256 * 256
    E, V, S = n_edges, n_kept, n_rhs
    Sv = (S + 7) // 8 * 8 if ts == 4 else S  # FP32 PCG vectors: samples padded to 8
    parts = [n_dofs * S * ts, 8, 8, 8, 8 * E, 8 * E, 8 * V, 16 * E] + [Sv * V * ts] * 4
    parts += [V * ts] + ([8 * E, 8 * V, 16 * E] + [Sv * V * 4] * 4 if ts == 4 else [])
    parts += [4 * S, 24, 4 * ts * E]
    return sum(up(x) for x in parts)


def test_noalloc_scratch_counts_the_sweep_constants():
    # a mixed-precision graph with long edges (node-parallel condensation);
    # the reported need must include the sweep constants of every edge
    G = _long_graph()
    for precision, ts in (("mixed", 4), ("fp64", 8)):
        opts = grf.make_options(precision)
        n_rhs = (16 << 20) // (ts * G.n_dofs) + 1
        with pytest.raises(grf.GrfError) as ei:
            grf.grf_vertex_solve_noalloc(G.handle, 1.7, 1.0, 0.5, n_rhs, 1, 1, 1, opts, stream=0)
        msg = str(ei.value)
        need = int(msg.split("needs ")[1].split(" bytes")[0])
        assert need == _scratch_bytes(G.n_dofs, G.n_kept, G.n_edges, n_rhs, ts), msg


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    G = _graph()
    opts = grf.make_options("fp64")
    n_rhs = (16 << 20) // (8 * G.n_dofs) + 1
    with pytest.raises(grf.GrfError) as ei:
        grf.grf_vertex_solve_noalloc(G.handle, 1.7, 1.0, 0.5, n_rhs, 1, 1, 1, opts, stream=0)
    assert ei.value.code == grf.GRF_EINVAL and "static scratch" in str(ei.value)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_allocating_vertex_solve(precision):
    import torch

    G = _graph()
    kappa, alpha, n_rhs = 1.7, 1.0, 5
    gen = torch.Generator(device="cpu").manual_seed(4)
    opts = grf.make_options(precision)
    for gamma in (0.05, 3.0):
        rhs = torch.randn((n_rhs, G.n_dofs), generator=gen, dtype=torch.float64).cuda()
        # the allocating entry point also makes the graph resident on the device
        g_ref, u_ref, _ = G.vertex_solve(kappa, alpha, gamma, rhs, precision=precision)
        for _call in range(2):
            g_out = torch.full((n_rhs, G.n_kept), float("nan"), dtype=torch.float64, device="cuda")
            u_out = torch.full_like(g_out, float("nan"))
            st = grf.grf_vertex_solve_noalloc(G.handle, kappa, alpha, gamma, n_rhs,
                                              rhs.data_ptr(), g_out.data_ptr(), u_out.data_ptr(),
                                              opts)
            assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0
            for got, ref in ((g_out, g_ref), (u_out, u_ref)):
                err = (torch.linalg.norm(got - ref, dim=1) / torch.linalg.norm(ref, dim=1)).max()
                assert float(err) < TOL[precision], float(err)


@pytest.mark.gpu
def test_noalloc_needs_a_resident_graph():
    import torch

    G = _graph()  # never used on the device
    out = torch.empty((1, G.n_kept), dtype=torch.float64, device="cuda")
    rhs = torch.zeros((1, G.n_dofs), dtype=torch.float64, device="cuda")
    with pytest.raises(grf.GrfError) as ei:
        grf.grf_vertex_solve_noalloc(G.handle, 1.0, 1.0, 1.0, 1, rhs.data_ptr(), out.data_ptr(),
                                     out.data_ptr(), grf.make_options("fp64"))
    assert ei.value.code == grf.GRF_EINVAL and "resident" in str(ei.value)


@pytest.mark.gpu
@pytest.mark.parametrize("sweep", ["auto", "nodes", "segments"])
@pytest.mark.parametrize("n_rhs", [4, 5])
def test_noalloc_long_edges_match_oracle(sweep, n_rhs):
    """Mixed precision on edges of 152-767 interior nodes, so that the
    node-parallel condensation (sweep auto or nodes) reads its sweep constants
    from the static array; against the oracle's global condensation and the
    allocating entry point, on two calls in a row."""
    import torch
    from oracle import fem, noise, sampler

    g = _long_graph_input()
    G = _long_graph()
    m = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=LONG_H)
    kappa, alpha = 1.7, 1.0
    ml, _, kmat = sampler.assemble(m, kappa)
    opts = grf.make_options("mixed", sweep=sweep)
    for gamma in (0.05, 3.0):
        rhs_np = noise.white_noise(ml, 11, n_rhs)
        rhs = torch.tensor(rhs_np, device="cuda")
        g_ref, u_ref = sampler.vertex_condensation(m, ml, kmat, gamma, rhs_np)
        g_al, u_al, _ = G.vertex_solve(kappa, alpha, gamma, rhs, precision="mixed")
        for _call in range(2):
            g_out = torch.full((n_rhs, G.n_kept), float("nan"), dtype=torch.float64, device="cuda")
            u_out = torch.full_like(g_out, float("nan"))
            st = grf.grf_vertex_solve_noalloc(G.handle, kappa, alpha, gamma, n_rhs,
                                              rhs.data_ptr(), g_out.data_ptr(), u_out.data_ptr(),
                                              opts)
            assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0
            for got, ref in ((g_out, g_ref), (u_out, u_ref), (g_out, g_al.cpu().numpy()),
                             (u_out, u_al.cpu().numpy())):
                got = got.cpu().numpy()
                err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
                assert err.max() < TOL["mixed"], err
