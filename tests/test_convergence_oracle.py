"""Pins of the oracle's convergence study (Sec. 4.1 strong error, Sec. 4.2
covariance error, Table 1) on a small synthetic metric graph: the nested-mesh
interpolation and noise projection against what they must preserve, and the
measured rates against the theory the paper quotes (strong 2 beta - 1/2,
covariance min(4 beta - 1/2, 2), for beta in (1/4, 1); Table 1 prints 0.51
and 1.00 for beta = 1/2 and 3/4, and 1.59 for the covariance at beta = 1/2)."""
import numpy as np
import pytest

import grf_inputs as gi
from oracle import convergence as cv
from oracle import fem


def _graph():
    # a triangle of unit edges and a pendant edge of length 1/2
    g = gi.Graph(4, np.array([0, 1, 2, 2]), np.array([1, 2, 0, 3]),
                 np.array([1.0, 1.0, 1.0, 0.5]))
    return g, np.array([2, 2, 2, 1])


def _positions(m: fem.Mesh):
    """Arc-length position of every DOF along its edge (vertices: 0) and the
    edge of every interior DOF."""
    x = np.zeros(m.n_dofs)
    edge = -np.ones(m.n_dofs, np.int64)
    for e in range(m.edge_u.shape[0]):
        for p in range(1, int(m.n_elems[e])):
            d = m.n_vertices + int(m.interior_offsets[e]) + p - 1
            x[d] = p * m.h_e[e]
            edge[d] = e
    return x, edge


def test_prolongation_interpolates_edgewise_linear_functions():
    g, base = _graph()
    mc, mf = cv.nested_mesh(g, base, 1), cv.nested_mesh(g, base, 3)
    P = cv.prolongation(mc, mf)
    # a continuous function, affine along every edge: vertex values plus
    # a(e) (x - x_u) ... realised by interpolating vertex values linearly
    rng = np.random.default_rng(0)
    fv = rng.standard_normal(mc.n_vertices)

    def sample(m):
        x, edge = _positions(m)
        f = np.zeros(m.n_dofs)
        f[:m.n_vertices] = fv
        for d in range(m.n_vertices, m.n_dofs):
            e = edge[d]
            s = x[d] / m.lengths[e]
            f[d] = (1 - s) * fv[m.edge_u[e]] + s * fv[m.edge_v[e]]
        return f

    np.testing.assert_allclose(P @ sample(mc), sample(mf), rtol=0, atol=1e-14)
    # rows sum to one, so the projection P^T keeps the total of the noise
    np.testing.assert_allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, atol=1e-14)
    w = rng.standard_normal(mf.n_dofs)
    assert abs((P.T @ w).sum() - w.sum()) < 1e-12


def test_projected_noise_has_the_coarse_consistent_mass_as_covariance():
    # Cov(P^T W_f) = P^T M_f P; with the fine consistent mass this is the coarse
    # consistent mass exactly (Galerkin identity of nested P1 spaces)
    g, base = _graph()
    mc, mf = cv.nested_mesh(g, base, 1), cv.nested_mesh(g, base, 3)
    P = cv.prolongation(mc, mf)
    lhs = (P.T @ fem.consistent_mass(mf) @ P).toarray()
    np.testing.assert_allclose(lhs, fem.consistent_mass(mc).toarray(), rtol=0, atol=1e-14)


@pytest.mark.parametrize("beta", [0.5, 0.75])
def test_strong_rate_matches_theory(beta):
    g, base = _graph()
    hs, errs = cv.strong_errors(g, base, [2, 3, 4, 5], 9, beta, 1.0, 100, 7)
    np.testing.assert_allclose(hs, 2.0 ** -np.arange(3, 7))
    assert np.all(np.diff(errs) < 0)
    assert abs(cv.rate(hs, errs) - (2 * beta - 0.5)) < 0.06


def test_covariance_rate_matches_theory():
    g, base = _graph()
    hs, errs = cv.covariance_errors(g, base, [1, 2, 3, 4], 7, 0.5, 1.0)
    assert np.all(np.diff(errs) < 0)
    assert abs(cv.rate(hs, errs) - 1.5) < 0.1
