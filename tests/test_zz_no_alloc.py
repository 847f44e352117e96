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
