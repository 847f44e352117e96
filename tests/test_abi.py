"""The C ABI library loads, exports every symbol include/grf.h declares, and its
host-side graph logic (validation, mesh, DOF map) agrees with the oracle's.
No device work: runs without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import grf_inputs as gi
import paper_2605_02670_gb300 as grf
from oracle import fem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "grf.h")).read()
    return sorted(set(re.findall(r"^\S.*?\b(grf_\w+)\(", src, re.M)))


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert "grf_sample" in names and "grf_graph_create" in names
    lib = ctypes.CDLL(grf.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(grf.C_SYMBOLS)


@pytest.mark.parametrize("name", ["square5", "rgg_small", "grid_small", "ba_small", "parts"])
def test_mesh_and_dof_map_match_oracle(name):
    if name == "parts":
        g = gi.disjoint_union(gi.grid_deleted(12, 12, 0.15, seed=3),
                              gi.random_small_graph(30, 40, 5), gi.interval(0.8), seed=3)
        h, clip = 2.0 ** -4, None
    elif name == "square5":
        g, h, clip = gi.square_diagonal(0), 2.0 ** -7, None
    elif name == "rgg_small":
        g, h, clip = gi.random_geometric(300, 0.07, seed=2), 2.0 ** -6, None
    elif name == "grid_small":
        g, h, clip = gi.grid_deleted(20, 20, 0.15, seed=7), 2.0 ** -4, None
    else:
        g, h, clip = gi.barabasi_albert(500, 3, seed=1), 2.0 ** -5, (2, 64)
    ne = grf.mesh_elements(g.lengths, h, clip)
    G = grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, n_elems=ne)
    m = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=h, clip=clip)
    assert G.n_dofs == m.n_dofs and G.n_kept == m.n_vertices and G.n_interior == m.n_interior
    np.testing.assert_array_equal(G.vertex_map, m.vertex_map)
    np.testing.assert_array_equal(G.interior_offsets, m.interior_offsets)
    G2 = grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=h)
    if clip is None:
        assert G2.n_dofs == m.n_dofs


@pytest.mark.parametrize("name", ["rgg", "parts"])
def test_vertex_order_is_a_banded_permutation(name):
    """The sample-group PCG's slot order (reverse Cuthill-McKee): a permutation
    of the kept vertices, a narrower bandwidth than the input numbering, and
    every connected component in one contiguous range of slots."""
    if name == "rgg":
        g = gi.random_geometric(400, 0.06, seed=3)
    else:
        g = gi.disjoint_union(gi.grid_deleted(15, 15, 0.15, seed=1),
                              gi.random_small_graph(40, 60, 2), gi.interval(0.5), seed=4)
    G = grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=0.1)
    perm = G.vertex_order
    n = G.n_kept
    np.testing.assert_array_equal(np.sort(perm), np.arange(n))
    slot = np.empty(n, np.int64)
    slot[perm] = np.arange(n)
    u, v = G.vertex_map[g.edge_u], G.vertex_map[g.edge_v]
    assert (u >= 0).all() and (v >= 0).all()
    assert np.abs(slot[u] - slot[v]).max() < np.abs(u - v).max() / 2
    comp = gi._components(n, u, v)
    for c in np.unique(comp):
        s = np.sort(slot[comp == c])
        assert s[-1] - s[0] + 1 == s.size


def test_disjoint_union_keeps_the_parts_as_components():
    parts = [gi.grid_deleted(10, 10, 0.15, seed=2), gi.random_small_graph(25, 35, 4),
             gi.interval(0.8)]
    g = gi.disjoint_union(*parts, seed=11)
    assert g.n_vertices == sum(p.n_vertices for p in parts)
    assert g.edge_u.shape[0] == sum(p.edge_u.shape[0] for p in parts)
    np.testing.assert_array_equal(np.sort(g.lengths),
                                  np.sort(np.concatenate([p.lengths for p in parts])))
    comp = gi._components(g.n_vertices, g.edge_u, g.edge_v)
    sizes = sorted(np.unique(comp, return_counts=True)[1].tolist())
    assert sizes == sorted(p.n_vertices for p in parts)
    # the parts' ids interleave: the smallest part is not a block of consecutive ids
    small = np.flatnonzero(comp == comp[g.edge_u[-1]])
    assert small.size == 2 and small[1] - small[0] > 1


@pytest.mark.parametrize("case,msg", [
    (([0], [0], [1.0], 2, 0.1), "self-loop"),
    (([0], [5], [1.0], 2, 0.1), "out of range"),
    (([0], [1], [-1.0], 2, 0.1), "length"),
    (([0], [1], [np.nan], 2, 0.1), "length"),
    (([0], [1], [1.0], 2, 0.0), "h > 0"),
])
def test_invalid_graphs_rejected(case, msg):
    with pytest.raises(grf.GrfError) as ei:
        grf.Graph(*case[:4], h=case[4])
    assert ei.value.code == grf.GRF_EINVAL and msg in str(ei.value)


def test_invalid_element_counts_rejected():
    with pytest.raises(grf.GrfError):
        grf.Graph([0], [1], [1.0], 2, n_elems=[0])


def test_invalid_sampling_parameters_rejected_before_device_work():
    G = grf.Graph([0, 1], [1, 2], [1.0, 0.5], 3, h=0.1)
    opts = grf.make_options("fp64")
    for kappa, beta, k in [(0.0, 0.5, 0.3), (1.0, 0.0, 0.3), (1.0, 0.5, 0.0), (np.nan, 0.5, 0.3)]:
        with pytest.raises(grf.GrfError) as ei:
            grf.grf_sample(G.handle, kappa, beta, k, 1, 2, 0, opts, stream=0)
        assert ei.value.code == grf.GRF_EINVAL
    bad = grf.grf_options(7, 0, 0, 0, 0.0)
    with pytest.raises(grf.GrfError):
        grf.grf_sample(G.handle, 1.0, 0.5, 0.3, 1, 2, 0, bad, stream=0)
    unsupported = grf.grf_options(0, 3, 0, 0, 0.0)
    with pytest.raises(grf.GrfError) as ei:
        grf.grf_sample(G.handle, 1.0, 0.5, 0.3, 1, 2, 0, unsupported, stream=0)
    assert ei.value.code == grf.GRF_ENOTSUP


def test_workspace_query_is_host_only():
    G = grf.Graph([0, 1], [1, 2], [1.0, 0.5], 3, h=0.1)
    b1 = G.workspace_bytes(0.75, 0.5, 4)
    b2 = G.workspace_bytes(0.75, 0.5, 8)
    b3 = G.workspace_bytes(1.75, 0.5, 8)
    assert 0 < b1 < b2 < b3


def test_weights_file_header_is_checked_before_device_work(tmp_path):
    """grf_precond_load rejects anything but a version-1 weights file of this
    network without touching the device."""
    g = gi.square_diagonal(0)
    G = grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=0.1)
    header = bytearray(48)
    header[:8] = b"GRFLPBB1"
    vals = np.array([1, grf.GRF_LP_PARAMS, 8, 64, 3, 1], np.int32).tobytes()
    header[8:8 + len(vals)] = vals
    body = np.zeros(grf.GRF_LP_PARAMS, np.float32).tobytes()
    cases = {
        "short": bytes(header) + body[:100],
        "magic": b"XXXXXXXX" + bytes(header[8:]) + body,
        "version": bytes(header[:8]) + np.int32(2).tobytes() + bytes(header[12:]) + body,
        "width": bytes(header[:20]) + np.int32(32).tobytes() + bytes(header[24:]) + body,
        "trailing": bytes(header) + body + b"\0",
    }
    for name, blob in cases.items():
        p = os.path.join(tmp_path, name + ".bin")
        with open(p, "wb") as f:
            f.write(blob)
        with pytest.raises(grf.GrfError) as ei:
            G.precond_load(p)
        assert ei.value.code == grf.GRF_EINVAL, name
    with pytest.raises(grf.GrfError):
        G.precond_load(os.path.join(tmp_path, "missing.bin"))


def test_learned_options_rejected_without_weights_or_in_fp64():
    g = gi.square_diagonal(0)
    G = grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=0.1)
    with pytest.raises(grf.GrfError) as ei:
        G.workspace_bytes(0.7, 0.5, 4, precision="fp64", precond="learned")
    assert ei.value.code == grf.GRF_ENOTSUP
    assert G.workspace_bytes(0.7, 0.5, 4, precision="mixed", precond="learned") > \
        G.workspace_bytes(0.7, 0.5, 4, precision="mixed")
    with pytest.raises(grf.GrfError) as ei:
        G.precond_get()
    assert ei.value.code == grf.GRF_EINVAL


def test_interior_and_sweep_options_checked_before_device_work():
    G = grf.Graph([0, 1], [1, 2], [1.0, 0.5], 3, h=0.1)
    bad_sweep = grf.make_options("mixed")
    bad_sweep.sweep = 7
    with pytest.raises(grf.GrfError) as ei:
        grf.grf_sample(G.handle, 1.0, 0.5, 0.3, 1, 2, 0, bad_sweep, stream=0)
    assert ei.value.code == grf.GRF_EINVAL
    bad_interior = grf.make_options("mixed")
    bad_interior.interior = 9
    with pytest.raises(grf.GrfError) as ei:
        grf.grf_sample(G.handle, 1.0, 0.5, 0.3, 1, 2, 0, bad_interior, stream=0)
    assert ei.value.code == grf.GRF_EINVAL
    for interior in ("spectral", "spectral_tc", "spectral_umma"):  # FP32 only
        with pytest.raises(grf.GrfError) as ei:
            grf.grf_sample(G.handle, 1.0, 0.5, 0.3, 1, 2, 0,
                           grf.make_options("fp64", interior=interior), stream=0)
        assert ei.value.code == grf.GRF_ENOTSUP
    # the consistent mass (the comparison system): mixed precision, Jacobi and
    # the tensor-core sine path only; unknown mass values are invalid
    bad_mass = grf.make_options("mixed")
    bad_mass.mass = 5
    with pytest.raises(grf.GrfError) as ei:
        grf.grf_sample(G.handle, 1.0, 0.5, 0.3, 1, 2, 0, bad_mass, stream=0)
    assert ei.value.code == grf.GRF_EINVAL
    for kw in ({"precision": "fp64"}, {"precision": "mixed", "interior": "thomas"},
               {"precision": "mixed", "interior": "spectral_tc"},
               {"precision": "mixed", "precond": "neumann"}):
        with pytest.raises(grf.GrfError) as ei:
            grf.grf_sample(G.handle, 1.0, 0.5, 0.3, 1, 2, 0,
                           grf.make_options(mass="consistent", **kw), stream=0)
        assert ei.value.code == grf.GRF_ENOTSUP
    assert grf.make_options("mixed", interior="spectral_tc", sweep="nodes").knobs() == {
        "pcg_layout": "auto", "recover_sg": 0, "interior": "spectral_tc", "sweep": "nodes"}


def test_timing_mask_checked_before_device_work():
    G = grf.Graph([0, 1], [1, 2], [1.0, 0.5], 3, h=0.1)
    assert grf.make_options("mixed", timing=True).timing == 1
    assert grf.make_options("mixed", timing=False).timing == 0
    assert grf.make_options("mixed", timing=["pcg"]).timing == grf.GRF_TIMING_ONLY | (1 << 3)
    assert grf.make_options("mixed", timing=("noise", "recover")).timing == (
        grf.GRF_TIMING_ONLY | 1 | (1 << 4))
    for flag in (grf.GRF_TIMING_ONLY, grf.GRF_TIMING_ONLY | (1 << 8) | 1):
        bad = grf.make_options("mixed")
        bad.timing = flag
        with pytest.raises(grf.GrfError) as ei:
            grf.grf_sample(G.handle, 1.0, 0.5, 0.3, 1, 2, 0, bad, stream=0)
        assert ei.value.code == grf.GRF_EINVAL and "timing" in str(ei.value)


def test_header_constants_match_the_binding():
    src = open(os.path.join(ROOT, "include", "grf.h")).read()
    found = 0
    for name, shift, val in re.findall(r"^#define (GRF_\w+) (?:\(1 << (\d+)\)|(-?\d+))", src,
                                       re.M):
        if hasattr(grf, name):
            assert getattr(grf, name) == (1 << int(shift) if shift else int(val)), name
            found += 1
    assert found >= 20


def test_binding_without_the_library_fails_loudly(tmp_path):
    """No CPU fallback: a copy of the package without libgrf.so refuses to import."""
    import shutil
    import subprocess
    import sys

    pkg = tmp_path / "paper_2605_02670_gb300"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_2605_02670_gb300", "__init__.py"), pkg / "__init__.py")
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    r = subprocess.run([sys.executable, "-c", "import paper_2605_02670_gb300"], cwd=tmp_path,
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "no CPU fallback" in r.stderr
