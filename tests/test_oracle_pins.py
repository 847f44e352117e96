"""Pins of the FP64 CPU oracle against facts that do not come from the oracle:
published known answers, the paper's printed entries and table values, closed
forms, dense eigen-decompositions and Monte-Carlo moments. CPU only."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.stats as st

import grf_inputs as gi
from oracle import fem, noise, philox, quadrature, sampler

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------- Philox


def test_philox_known_answers():
    for r in _rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(np.array(v[:4], np.uint32), np.array(v[4:6], np.uint32))
        assert [int(x) for x in out] == v[6:10]


def test_noise_counter_layout():
    # word j of sample s is word j%4 of the block with counter (j//4, 0, s, 0)
    seed = 0x1234_5678_9ABC_DEF0
    w = philox.noise_words(seed, 11, 3)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    for s in range(3):
        for j in (0, 3, 4, 10):
            blk = philox.philox4x32_10(np.array([j // 4, 0, s, 0], np.uint32), key)
            assert w[s, j] == blk[j % 4]


# ---------------------------------------------------------------- noise


def test_uniform_and_box_muller_special_values():
    u = noise.uniforms(np.array([0, 0xFFFFFFFF], np.uint32))
    assert u[0] == 2.0 ** -33 and u[1] == 1.0 - 2.0 ** -33
    # u_a = e^{-1/2} gives r = 1; u_b = 1/4 and 1/8 give angles pi/2 and pi/4
    z = noise.box_muller(np.array([math.exp(-0.5), 0.25, math.exp(-0.5), 0.125]))
    np.testing.assert_allclose(z, [0.0, 1.0, math.sqrt(0.5), math.sqrt(0.5)], atol=1e-15)


def test_standard_normals_distribution():
    xi = noise.standard_normals(7, 50_000, 2).ravel()
    assert abs(xi.mean()) < 5 / math.sqrt(xi.size)
    assert abs(xi.var() - 1) < 5 * math.sqrt(2 / xi.size)
    assert st.kstest(xi, "norm").pvalue > 1e-4
    # the two normals of one Box-Muller pair are uncorrelated
    assert abs(np.corrcoef(xi[0::2], xi[1::2])[0, 1]) < 5 / math.sqrt(xi.size / 2)


# ---------------------------------------------------------------- mesh and matrices


def test_mesh_counts_match_paper_table():
    """Sec. 4.3 table: N = 63 |E| for BA(n, 2) graphs with unit lengths at h = 2^-6."""
    for n, n_tab in _rows("table_interior_counts.txt"):
        n, n_tab = int(n), int(n_tab)
        if n > 5000:
            continue  # the generator is pure Python; the count rule is the same
        g = gi.barabasi_albert(n, 2, seed=3, lengths="unit")
        assert g.n_edges == 2 * (n - 2)
        m = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=2.0 ** -6)
        assert m.n_interior == n_tab
        assert m.n_dofs == n + n_tab  # Phase 1: N = |V| + sum (N_e - 2)


def test_mass_and_stiffness_entries_match_paper():
    """Entries printed in Sec. 3, Phase 2 (lumped mass and stiffness), on a
    star with three edges (one vertex of degree 3) and a parallel edge."""
    g = gi.Graph(4, np.array([0, 0, 0, 1]), np.array([1, 2, 3, 2]),
                 np.array([0.7, 1.1, 0.45, 0.9]))
    m = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, 4, h=0.1)
    ml = fem.lumped_mass(m)
    gm = fem.stiffness(m).toarray()
    cm = fem.consistent_mass(m).toarray()
    he = m.h_e
    for v in range(4):
        inc = [e for e in range(4) if v in (g.edge_u[e], g.edge_v[e])]
        assert ml[v] == pytest.approx(sum(he[e] / 2 for e in inc), rel=1e-14)
        assert gm[v, v] == pytest.approx(sum(1 / he[e] for e in inc), rel=1e-14)
        assert cm[v, v] == pytest.approx(sum(he[e] / 3 for e in inc), rel=1e-14)
    for e in range(4):
        o = m.n_vertices + m.interior_offsets[e]
        mi = m.n_elems[e] - 1
        for i in range(mi):
            assert ml[o + i] == pytest.approx(he[e], rel=1e-14)
            assert gm[o + i, o + i] == pytest.approx(2 / he[e], rel=1e-14)
            assert cm[o + i, o + i] == pytest.approx(2 * he[e] / 3, rel=1e-14)
            if i + 1 < mi:
                assert gm[o + i, o + i + 1] == pytest.approx(-1 / he[e], rel=1e-14)
        # vertex - adjacent interior couplings
        assert gm[g.edge_u[e], o] == pytest.approx(-1 / he[e], rel=1e-14)
        assert gm[g.edge_v[e], o + mi - 1] == pytest.approx(-1 / he[e], rel=1e-14)
        assert cm[g.edge_v[e], o + mi - 1] == pytest.approx(he[e] / 6, rel=1e-14)
    # lumped = row sums of consistent (Sec. 2.5); total mass = total length
    np.testing.assert_allclose(ml, cm.sum(axis=1), rtol=1e-14)
    assert ml.sum() == pytest.approx(g.lengths.sum(), rel=1e-14)
    np.testing.assert_allclose(gm.sum(axis=1), 0, atol=1e-9)


def test_degree_zero_vertices_dropped():
    g = gi.Graph(5, np.array([0, 3]), np.array([3, 4]), np.array([1.0, 1.0]))
    m = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, 5, h=0.25)
    assert list(m.vertex_map) == [0, -1, -1, 1, 2]
    assert m.n_dofs == 3 + 2 * 3


# ---------------------------------------------------------------- quadrature


def test_quadrature_limits_and_coefficients():
    assert quadrature.limits(0.75, 0.5) == (14, 40)
    assert quadrature.limits(0.25, 0.3) == (110, 37)
    c_i, c_l = quadrature.coefficients(0.6, 0.4)
    km, kp = quadrature.limits(0.6, 0.4)
    y = np.arange(-km, kp + 1) * 0.4
    np.testing.assert_allclose(c_i, math.pi / (2 * 0.4 * math.sin(0.6 * math.pi)) * np.exp(-1.2 * y))
    np.testing.assert_allclose(c_l / c_i, np.exp(2 * y))


@pytest.mark.parametrize("beta", [0.25, 0.5, 0.75, 0.9])
def test_quadrature_reproduces_fractional_power(beta):
    """sum_l (c_I + c_L lambda)^{-1} -> lambda^{-beta} (Eq. 2 is exact); with
    k = 0.2 the sinc rule is accurate to ~1e-8 on [1, 1e4]."""
    lam = np.logspace(0, 4, 300)
    rel = np.abs(quadrature.scalar(lam, beta, 0.2) * lam ** beta - 1)
    assert rel.max() < 1e-7


# ---------------------------------------------------------------- whole sampler, closed forms


def _interval_closed_form(n, length, kappa, b, qfun):
    """One edge, two degree-1 vertices: Kirchhoff reduces to Neumann. Lumped
    P1 eigenpairs: v_j(i) = cos(j pi i / n), lambda_j = kappa^2 + 4/h^2
    sin^2(j pi / (2n)). Returns U in the sampler's DOF order."""
    h = length / n
    i = np.arange(n + 1)
    j = np.arange(n + 1)
    v = np.cos(np.pi * np.outer(i, j) / n)          # [pos, j]
    mlp = np.full(n + 1, h)
    mlp[0] = mlp[-1] = h / 2
    lam = kappa ** 2 + 4 / h ** 2 * np.sin(j * np.pi / (2 * n)) ** 2
    order = np.concatenate([[0, n], np.arange(1, n)])  # DOF index -> position
    bp = np.zeros_like(b)
    bp[:, order] = b
    nu = (v * v * mlp[:, None]).sum(axis=0)
    coef = (bp @ v) / nu * qfun(lam)
    up = coef @ v.T
    return up[:, order]


@pytest.mark.parametrize("beta", [0.3, 0.75, 1.0, 1.25, 2.0])
def test_single_interval_closed_form(beta):
    kappa, k, n, length = 3.0, 0.4, 37, 1.3
    g = gi.interval(length)
    mesh, u, b = sampler.sample(g, kappa, beta, k, seed=5, n_samples=3, n_elems=[n])
    nint = math.floor(beta)
    f = beta - nint
    if f < 1e-12:
        q = lambda lam: lam ** (-float(nint))
    else:
        q = lambda lam: quadrature.scalar(lam, f, k) * lam ** (-float(nint))
    ref = _interval_closed_form(n, length, kappa, b, q)
    np.testing.assert_allclose(u, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def _dense_fractional(mesh, kappa, b, qfun):
    ml = fem.lumped_mass(mesh)
    kd = (kappa ** 2 * np.diag(ml) + fem.stiffness(mesh).toarray())
    lam, vec = sla.eigh(kd, np.diag(ml))       # K v = lam M_L v, v^T M_L v = 1
    return ((b @ vec) * qfun(lam)) @ vec.T


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_graph_against_dense_eigendecomposition(seed):
    g = gi.random_small_graph(7, 11, seed)
    kappa, beta, k = 2.0, 0.6, 0.35
    mesh, u, b = sampler.sample(g, kappa, beta, k, seed=9, n_samples=2, h=0.15)
    ref = _dense_fractional(mesh, kappa, b, lambda lam: quadrature.scalar(lam, beta, k))
    np.testing.assert_allclose(u, ref, rtol=1e-9, atol=1e-11 * np.abs(ref).max())
    # and the quadrature itself is close to the exact fractional power
    exact = _dense_fractional(mesh, kappa, b, lambda lam: lam ** -beta)
    assert np.abs(u - exact).max() < 2e-2 * np.abs(exact).max()


def test_half_powers_compose_to_the_stiffness_solve():
    """Two applications of the beta = 1/2 quadrature with the lumped mass between
    them give one solve with K: with L = M_L^-1 K, each application is
    L^-1/2 M_L^-1 up to q(lambda) lambda^1/2 - 1 per mode, so the composition is
    K^-1 b up to q(lambda)^2 lambda - 1, below about 2e-7 here (k = 0.2, spectrum
    inside [2.25, 713] for kappa = 1.5 and elements of at least 0.075). The
    consistent mass in place of M_L between the two breaks it."""
    g = gi.random_small_graph(9, 14, 5)
    mesh = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=0.1)
    ml, _, kmat = sampler.assemble(mesh, 1.5)
    b = np.random.default_rng(3).standard_normal((2, mesh.n_dofs))
    ref = sampler.stiff_solve(kmat, b)

    def rel(u):
        return np.sqrt((ml * (u - ref) ** 2).sum()) / np.sqrt((ml * ref ** 2).sum())

    half = sampler.fractional_apply(ml, kmat, b, 0.5, 0.2)
    assert rel(sampler.fractional_apply(ml, kmat, ml[None, :] * half, 0.5, 0.2)) < 3e-7
    mc = fem.consistent_mass(mesh)
    wrong = sampler.fractional_apply(ml, kmat, np.asarray((mc @ half.T).T), 0.5, 0.2)
    assert rel(wrong) > 1e-3


def test_kirchhoff_and_continuity_at_vertices():
    """u is continuous by construction (one DOF per vertex). The vertex rows
    of (M_L + t K) u - b are the discrete Kirchhoff balance: zero flux sum up
    to the mass term. Checked with the paper's printed stiffness entries."""
    g = gi.random_small_graph(6, 9, 4)
    mesh = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, 6, h=0.2)
    ml, _, kmat = sampler.assemble(mesh, 1.5)
    b = noise.white_noise(ml, 3, 1)
    t = 0.7
    u = sampler.shifted_sum(ml, kmat, b, [t], [1.0])[0]
    for v in range(mesh.n_vertices):
        flux = 0.0
        mass = 0.0
        for e in range(g.n_edges):
            he = mesh.h_e[e]
            o = mesh.n_vertices + mesh.interior_offsets[e]
            if mesh.edge_u[e] == v:
                nb = o if mesh.n_elems[e] > 1 else mesh.edge_v[e]
            elif mesh.edge_v[e] == v:
                nb = o + mesh.n_elems[e] - 2 if mesh.n_elems[e] > 1 else mesh.edge_u[e]
            else:
                continue
            flux += (u[v] - u[nb]) / he          # outward difference quotient
            mass += he / 2
        lhs = mass * (1 + t * 1.5 ** 2) * u[v] + t * flux
        assert lhs == pytest.approx(b[0, v], rel=1e-9, abs=1e-12)


def test_sample_covariance_matches_exact_fem_covariance():
    """Cov(U) = Q M_L Q^T with Q = sum_l w_l (M_L + t_l K)^{-1}: the noise has
    covariance M_L (Sec. 2.4-2.5). 20000 samples on a small graph."""
    g = gi.Graph(3, np.array([0, 1]), np.array([1, 2]), np.array([0.6, 0.9]))
    kappa, beta, k, s = 2.0, 0.75, 0.5, 20000
    mesh, u, _ = sampler.sample(g, kappa, beta, k, seed=11, n_samples=s, h=0.2)
    ml, _, kmat = sampler.assemble(mesh, kappa)
    t, w = quadrature.nodes(beta, k)
    q = sum(wl * np.linalg.inv(np.diag(ml) + tl * kmat.toarray()) for tl, wl in zip(t, w))
    cov = q @ np.diag(ml) @ q.T
    emp = np.cov(u.T)
    se = np.sqrt((np.outer(np.diag(cov), np.diag(cov)) + cov ** 2) / s)
    z = np.abs(emp - cov) / se
    assert z.max() < 5.0
    assert np.abs(emp.diagonal() / cov.diagonal() - 1).max() < 0.06


# ---------------------------------------------------------------- vertex condensation


def _edge_local_schur(he, n, alpha, t, kappa):
    """2x2 Schur block of one edge from the paper's local matrices (Eq.
    local_reduced_schur), by dense inversion of the interior block."""
    ml = np.full(n + 1, he)
    ml[0] = ml[-1] = he / 2
    gk = (np.diag(np.full(n + 1, 2.0)) - np.eye(n + 1, k=1) - np.eye(n + 1, k=-1)) / he
    gk[0, 0] = gk[-1, -1] = 1 / he
    a = alpha * np.diag(ml) + t * (kappa ** 2 * np.diag(ml) + gk)
    bidx = [0, n]
    iidx = list(range(1, n))
    if not iidx:
        return a[np.ix_(bidx, bidx)]
    return a[np.ix_(bidx, bidx)] - a[np.ix_(bidx, iidx)] @ np.linalg.solve(
        a[np.ix_(iidx, iidx)], a[np.ix_(iidx, bidx)])


def test_vertex_condensation_against_edge_local_assembly():
    g = gi.random_small_graph(5, 8, 6)
    kappa = 1.7
    mesh = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, 5, h=0.17)
    ml, _, kmat = sampler.assemble(mesh, kappa)
    b = noise.white_noise(ml, 2, 2)
    for t in (1e-3, 0.5, 40.0):
        s_dense = np.zeros((5, 5))
        for e in range(g.n_edges):
            se = _edge_local_schur(mesh.h_e[e], mesh.n_elems[e], 1.0, t, kappa)
            idx = [mesh.edge_u[e], mesh.edge_v[e]]
            s_dense[np.ix_(idx, idx)] += se
        np.testing.assert_allclose(sampler.vertex_schur_dense(mesh, ml, kmat, t), s_dense,
                                   rtol=1e-10, atol=1e-12 * np.abs(s_dense).max())
        gv, uv = sampler.vertex_condensation(mesh, ml, kmat, t, b)
        np.testing.assert_allclose(uv, np.linalg.solve(s_dense, gv.T).T, rtol=1e-9)


def test_edge_schur_block_closed_form():
    """With 2 + delta = 2 cosh(theta), (T^{-1})_11 = sinh(m theta)/sinh((m+1) theta)
    and (T^{-1})_1m = sinh(theta)/sinh((m+1) theta) for T = tridiag(-1, 2+delta, -1)."""
    kappa = 2.5
    for length, n, t in [(1.0, 9, 0.3), (0.4, 33, 5e-4), (2.0, 1, 3.0), (1.5, 2, 80.0)]:
        g = gi.interval(length)
        mesh = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, 2, n_elems=[n])
        ml, _, kmat = sampler.assemble(mesh, kappa)
        s = sampler.vertex_schur_dense(mesh, ml, kmat, t)
        he = length / n
        c = t / he
        delta = (1 + t * kappa ** 2) * he ** 2 / t
        th = math.acosh(1 + delta / 2)
        m = n - 1
        saa = c * (1 + delta / 2 - math.sinh(m * th) / math.sinh((m + 1) * th))
        sab = -c * math.sinh(th) / math.sinh((m + 1) * th)
        np.testing.assert_allclose(s, [[saa, sab], [sab, saa]], rtol=1e-10)


# ---------------------------------------------------------------- planted mistakes


def test_planted_mistakes_are_caught(monkeypatch):
    """A wrong weight, a dropped kappa^2 or a wrong noise scale in the oracle
    makes the closed-form pins fail."""
    kappa, beta, k, n, length = 3.0, 0.75, 0.2, 20, 1.0
    g = gi.interval(length)
    q = lambda lam: lam ** -beta   # exact; the k = 0.2 rule is within ~1e-8 of it

    def err():
        mesh, u, b = sampler.sample(g, kappa, beta, k, seed=5, n_samples=2, n_elems=[n])
        ref = _interval_closed_form(n, length, kappa, b, q)
        return np.abs(u - ref).max() / np.abs(ref).max()

    assert err() < 1e-6
    good_nodes = quadrature.nodes
    monkeypatch.setattr(quadrature, "nodes", lambda b_, k_: (good_nodes(b_, k_)[0],
                                                             0.5 * good_nodes(b_, k_)[1]))
    assert err() > 0.1
    monkeypatch.setattr(quadrature, "nodes", good_nodes)
    good_assemble = sampler.assemble
    monkeypatch.setattr(sampler, "assemble",
                        lambda mesh, kap: good_assemble(mesh, 0.5 * kap))
    assert err() > 1e-2
