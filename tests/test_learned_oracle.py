"""Pins of the FP64 reference of the learned BB^T preconditioner (CPU only):
central finite differences of the loss, the Jacobi limit at initialisation,
positive definiteness, and the per-edge Schur blocks against global assembly."""
import numpy as np
import pytest

import grf_inputs as gi
from oracle import fem, learned, sampler


def _setup(seed=2, t=0.8, kappa=1.5):
    g = gi.random_small_graph(9, 15, seed)
    mesh = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, 9, h=0.2)
    suu, suv = sampler.edge_schur_blocks(mesh, kappa, t)
    diag = np.zeros(mesh.n_vertices)
    np.add.at(diag, mesh.edge_u, suu)
    np.add.at(diag, mesh.edge_v, suu)
    inc = learned.Incidence(mesh.n_vertices, mesh.edge_u, mesh.edge_v)
    a = learned.scaled_system(inc, diag, suv)
    x = learned.features(inc, a, t)
    return mesh, inc, a, x, diag, suu, suv


def _pairs(inc, a, n, seed):
    rng = np.random.default_rng(seed)
    V = inc.n_vertices
    S = np.eye(V)
    for k in range(len(a)):
        S[inc.src[k], inc.nbr[k]] -= a[k]
    E = rng.standard_normal((n, V))
    R = E @ S.T
    return R, E, S


def test_edge_blocks_sum_to_global_schur():
    kappa, t = 1.5, 0.8
    mesh, inc, a, x, diag, suu, suv = _setup(kappa=kappa, t=t)
    ml, _, kmat = sampler.assemble(mesh, kappa)
    s = sampler.vertex_schur_dense(mesh, ml, kmat, t)
    np.testing.assert_allclose(np.diag(s), diag, rtol=1e-10)
    dense = np.zeros_like(s)
    for e in range(len(suv)):
        dense[mesh.edge_u[e], mesh.edge_v[e]] += suv[e]
        dense[mesh.edge_v[e], mesh.edge_u[e]] += suv[e]
    off = ~np.eye(len(diag), dtype=bool)
    np.testing.assert_allclose(dense[off], s[off], rtol=1e-10, atol=1e-14)


def test_scaled_system_is_spd_with_unit_diagonal():
    mesh, inc, a, x, *_ = _setup()
    _, _, S = _pairs(inc, a, 1, 0)
    np.testing.assert_allclose(np.diag(S), 1.0)
    np.testing.assert_allclose(S, S.T, atol=1e-14)
    assert np.linalg.eigvalsh(S).min() > 0
    assert (a > 0).all()


def test_initial_network_is_jacobi():
    mesh, inc, a, x, *_ = _setup()
    p = learned.init_params(0)
    s, n, _ = learned.forward(p, inc, a, x)
    assert np.all(s == 0) and np.all(n == 0)
    R, E, S = _pairs(inc, a, 3, 1)
    loss, _ = learned.loss_and_grad(p, inc, a, x, R, E)
    ref = np.mean([(r - e) @ S @ (r - e) / (r @ e) for r, e in zip(R, E)])
    assert loss == pytest.approx(ref, rel=1e-12)


def test_gradient_against_central_differences():
    mesh, inc, a, x, *_ = _setup(seed=5)
    rng = np.random.default_rng(3)
    p = learned.init_params(4)
    for k in ("ws", "u", "up"):
        p[k] = 0.2 * rng.standard_normal(p[k].shape)
    p["cs"] = np.array(0.1)
    p["cn"] = np.array(-0.05)
    R, E, _ = _pairs(inc, a, 2, 7)
    _, g = learned.loss_and_grad(p, inc, a, x, R, E)
    flat = learned.flatten(p)
    gflat = learned.flatten(g)
    idx = np.unique(np.concatenate([rng.choice(flat.size, 60, replace=False),
                                    np.arange(flat.size - 194, flat.size)]))
    eps = 1e-6
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += eps
        fm[i] -= eps
        lp, _ = learned.loss_and_grad(learned.unflatten(fp), inc, a, x, R, E)
        lm, _ = learned.loss_and_grad(learned.unflatten(fm), inc, a, x, R, E)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gflat[i])


def test_preconditioner_is_symmetric_positive_definite():
    mesh, inc, a, x, *_ = _setup(seed=8)
    rng = np.random.default_rng(9)
    p = learned.init_params(1)
    for k in ("ws", "u", "up"):
        p[k] = 0.3 * rng.standard_normal(p[k].shape)
    s, n, _ = learned.forward(p, inc, a, x)
    V = inc.n_vertices
    P = np.stack([learned.precondition(inc, s, n, np.eye(V)[i]) for i in range(V)], axis=1)
    np.testing.assert_allclose(P, P.T, atol=1e-12)
    assert np.linalg.eigvalsh(P).min() > 0


def test_gradient_descent_lowers_the_loss():
    mesh, inc, a, x, *_ = _setup(seed=11)
    R, E, _ = _pairs(inc, a, 8, 2)
    p = learned.init_params(3)
    l0, _ = learned.loss_and_grad(p, inc, a, x, R, E)
    for _ in range(30):
        loss, g = learned.loss_and_grad(p, inc, a, x, R, E)
        for k in p:
            p[k] = p[k] - 0.02 * g[k]
    assert loss < 0.9 * l0
