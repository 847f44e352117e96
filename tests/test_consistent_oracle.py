"""Pins of the consistent-mass comparison system in the oracle (Sec. 2.4 Eq.
wh_def, Sec. 3 Phase 2 consistent case): the Cholesky noise against the
printed mass entries and its covariance, the sampler against the closed-form
eigenpairs of the consistent-mass pencil on one interval, and the edge blocks
of the consistent shifted matrix against the lumped ones with the transformed
constants delta' = delta / (1 - delta / 6), c' = c (1 - delta / 6)."""
import math

import numpy as np
import pytest

import grf_inputs as gi
from oracle import consistent, fem, noise, quadrature


def _mesh(g, h):
    return fem.build_mesh(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=h)


def test_cholesky_factor_reproduces_the_printed_mass_and_its_interior_pivots():
    g = gi.random_small_graph(6, 9, 2)
    m = _mesh(g, 0.2)
    r = consistent.cholesky_factor(m)
    perm = consistent.cholesky_order(m)
    mc = fem.consistent_mass(m).toarray()
    np.testing.assert_allclose(r @ r.T, mc[np.ix_(perm, perm)], rtol=0, atol=1e-15)
    # the interiors come first, edge by edge: an edge's block is tridiagonal
    # (2h/3, h/6), so its squared pivots follow p_1 = 2h/3,
    # p_{i+1} = 2h/3 - (h/6)^2 / p_i
    k = 0
    for e in range(m.edge_u.shape[0]):
        h = m.h_e[e]
        p = 2 * h / 3
        for i in range(int(m.n_elems[e]) - 1):
            assert r[k, k] ** 2 == pytest.approx(p, rel=1e-12)
            if i > 0:  # R R^T = M below the diagonal: r_(k, k-1) r_(k-1, k-1) = h/6
                assert r[k, k - 1] * r[k - 1, k - 1] == pytest.approx(h / 6, rel=1e-12)
            p = 2 * h / 3 - (h / 6) ** 2 / p
            k += 1


def test_cholesky_noise_has_the_consistent_mass_as_covariance():
    g = gi.square_diagonal(0)
    m = _mesh(g, 0.25)
    S = 40000
    w = consistent.white_noise(m, 9, S)
    cov = w.T @ w / S
    mc = fem.consistent_mass(m).toarray()
    # entrywise within 5 standard errors: var(w_i w_j) = M_ii M_jj + M_ij^2
    se = np.sqrt((np.outer(np.diag(mc), np.diag(mc)) + mc ** 2) / S)
    assert np.all(np.abs(cov - mc) < 5 * se)


@pytest.mark.parametrize("beta", [0.3, 0.75, 1.25])
def test_interval_matches_the_consistent_mass_eigenpairs(beta):
    n, length, kappa, k = 24, 1.7, 2.5, 0.3
    g = gi.interval(length)
    m = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, g.n_vertices, n_elems=[n])
    mc, _, kc = consistent.assemble(m, kappa)
    w = consistent.white_noise(m, 4, 3)
    u = consistent.fractional_apply(mc, kc, w, beta, k)
    # positions 0..n along the interval: vertex 0, the interiors, vertex 1
    pos = np.concatenate([[0], 2 + np.arange(n - 1), [1]])
    f = beta - math.floor(beta)
    if beta >= 1:  # (K^-1 M)^n applied to the fractional part: q(lam) lam^-n
        t, wq = quadrature.nodes(f, k)
        ref = np.zeros_like(w[:, pos])
        i = np.arange(n + 1)
        h = length / n
        mpos = np.zeros((n + 1, n + 1))
        for a in range(n):
            mpos[a:a + 2, a:a + 2] += h / 6 * np.array([[2.0, 1.0], [1.0, 2.0]])
        for j in range(n + 1):
            v = np.cos(j * math.pi * i / n)
            lam = kappa ** 2 + 6 * (1 - math.cos(j * math.pi / n)) / (
                h * h * (2 + math.cos(j * math.pi / n)))
            q = float((wq / (1 + t * lam)).sum()) * lam ** -math.floor(beta)
            ref += q * np.outer(w[:, pos] @ v, v) / float(v @ mpos @ v)
    else:
        ref = consistent.interval_closed_form(n, length, kappa, beta, k, w[:, pos])
    np.testing.assert_allclose(u[:, pos], ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_consistent_edge_blocks_are_lumped_blocks_with_transformed_constants():
    # one edge of m interior nodes: the consistent interior block of
    # alpha M + gamma (kappa^2 M + G) is c' tridiag(-1, 2 + delta', -1), the
    # vertex-interior coupling -c' and each end's vertex entry c' (1 + delta'/2),
    # with delta = (alpha / gamma + kappa^2) h^2, c = gamma / h
    n, h, kappa = 9, 0.13, 1.7
    g = gi.Graph(2, np.array([0]), np.array([1]), np.array([n * h]))
    m = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, g.n_vertices, n_elems=[n])
    mc = fem.consistent_mass(m).toarray()
    gm = fem.stiffness(m).toarray()
    for alpha, gamma in ((1.0, 1e-6), (1.0, h * h / 6 * 0.9), (1.0, 0.3), (0.0, 1.0)):
        a = alpha * mc + gamma * (kappa ** 2 * mc + gm)
        delta = (alpha / gamma + kappa ** 2) * h * h
        c = gamma / h
        cp = c * (1 - delta / 6)
        dp = delta / (1 - delta / 6)
        inner = a[2:, 2:]
        np.testing.assert_allclose(np.diag(inner), cp * (2 + dp), rtol=1e-12)
        np.testing.assert_allclose(np.diag(inner, 1), -cp, rtol=1e-12)
        assert a[0, 2] == pytest.approx(-cp, rel=1e-12)
        assert a[0, 0] == pytest.approx(cp * (1 + dp / 2), rel=1e-12)
