"""Learned B B^T preconditioner on the GPU (through the C ABI) against the FP64
oracle of oracle/learned.py.

Tolerances. The network's dense layers take BF16 operands (8 significant bits,
unit roundoff u = 2^-9 ~ 2e-3) with FP32 accumulation; the input features are
rounded to BF16 too. Each of the four layers adds a relative error of a few u
to its output, so the heads s and n agree with the FP64 forward pass to about
1e-2 in norm (bound 3e-2 below). The backward pass multiplies BF16-rounded
activations and upstream gradients again: gradient blocks to 6e-2 in norm and
a cosine similarity above 0.998 with the FP64 gradient. The preconditioned
sampler is held to the same field tolerance as the Jacobi path (1e-4, mixed
precision): the preconditioner changes how PCG converges, not what it
converges to."""
import os

import numpy as np
import pytest

import grf_inputs as gi
from oracle import fem, learned, sampler

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

grf = pytest.importorskip("paper_2605_02670_gb300")


def rel_l2(u, ref, ml):
    u = np.atleast_2d(u)
    ref = np.atleast_2d(ref)
    num = np.sqrt((ml[None, :] * (u - ref) ** 2).sum(axis=1))
    den = np.sqrt((ml[None, :] * ref ** 2).sum(axis=1))
    return float((num / den).max())


def make(g, h=None, n_elems=None):
    G = grf.Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=h, n_elems=n_elems)
    m = fem.build_mesh(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=h, n_elems=n_elems)
    return G, m


def oracle_system(m, kappa, alpha, gamma):
    """Scaled vertex system of A = alpha M_L + gamma K in the oracle's terms."""
    t = gamma / alpha
    suu, suv = sampler.edge_schur_blocks(m, kappa, t)
    diag = np.zeros(m.n_vertices)
    np.add.at(diag, m.edge_u, suu)
    np.add.at(diag, m.edge_v, suu)
    inc = learned.Incidence(m.n_vertices, m.edge_u, m.edge_v)
    a = learned.scaled_system(inc, diag, suv)
    x = learned.features(inc, a, t)
    return inc, a, x


def random_heads(seed):
    rng = np.random.default_rng(seed)
    p = learned.init_params(seed)
    for k in ("ws", "u", "up"):
        p[k] = 0.2 * rng.standard_normal(p[k].shape)
    p["cs"] = np.array(0.1)
    p["cn"] = np.array(-0.05)
    return p


def dense_s_hat(inc, a):
    V = inc.n_vertices
    S = np.eye(V)
    np.add.at(S, (inc.src, inc.nbr), -a)
    return S


def nrel(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


GRAPH = lambda: (gi.random_small_graph(40, 75, 4), 0.12)


def test_parameter_count_matches_oracle():
    assert learned.n_params() == grf.GRF_LP_PARAMS


@pytest.mark.parametrize("t", [1e-3, 0.8, 40.0])
def test_forward_matches_oracle(t):
    g, h = GRAPH()
    G, m = make(g, h)
    kappa = 1.5
    p = random_heads(5)
    G.precond_set(learned.flatten(p).astype(np.float32))
    s_dev, n_dev = G.precond_forward(kappa, 1.0, t)
    inc, a, x = oracle_system(m, kappa, 1.0, t)
    s_ref, n_ref, _ = learned.forward(p, inc, a, x)
    assert nrel(s_dev, s_ref) < 3e-2
    assert nrel(n_dev, n_ref) < 3e-2


def test_zero_heads_give_identity():
    g, h = GRAPH()
    G, m = make(g, h)
    G.precond_init(3)
    s, n = G.precond_forward(2.0, 1.0, 0.5)
    assert np.all(s == 0) and np.all(n == 0)
    w = G.precond_get()
    pr = learned.unflatten(w.astype(np.float64))
    for k in ("ws", "cs", "u", "up", "cn", "b0", "b1", "b2", "b3"):
        assert np.all(pr[k] == 0), k
    # He scale of the layers
    assert abs(np.std(pr["W2"]) - np.sqrt(2.0 / 128)) < 0.01


def test_loss_and_gradient_match_oracle():
    g, h = GRAPH()
    G, m = make(g, h)
    kappa, t = 1.5, 0.8
    p = random_heads(7)
    G.precond_set(learned.flatten(p).astype(np.float32))
    inc, a, x = oracle_system(m, kappa, 1.0, t)
    S = dense_s_hat(inc, a)
    rng = np.random.default_rng(11)
    E = rng.standard_normal((6, inc.n_vertices))
    R = E @ S
    loss_dev, grad_dev = G.precond_loss_grad(kappa, 1.0, t, R, E)
    loss_ref, gref, heads = learned.loss_and_grad(p, inc, a, x, R, E, details=True)
    assert abs(loss_dev - loss_ref) < 3e-2 * loss_ref
    gd = learned.unflatten(grad_dev.astype(np.float64))
    for k in gref:
        ref = np.asarray(gref[k])
        if k == "cs":  # a sum over vertices with cancellation: bound by the sum of |terms|
            assert abs(gd[k] - ref) < 6e-2 * np.abs(heads["ds"]).sum()
        elif k == "cn":
            assert abs(gd[k] - ref) < 6e-2 * np.abs(a * heads["dn"]).sum()
        else:
            assert nrel(np.asarray(gd[k]), ref) < 6e-2, k
    gflat = learned.flatten(gref)
    cos = float(grad_dev @ gflat / (np.linalg.norm(grad_dev) * np.linalg.norm(gflat)))
    assert cos > 0.998


def test_save_load_roundtrip(tmp_path):
    g, h = GRAPH()
    G, _ = make(g, h)
    G2, _ = make(g, h)
    p = learned.flatten(random_heads(2)).astype(np.float32)
    G.precond_set(p)
    path = os.path.join(tmp_path, "w.bin")
    G.precond_save(path)
    G2.precond_load(path)
    np.testing.assert_array_equal(G2.precond_get(), p)
    assert os.path.getsize(path) == 48 + 4 * grf.GRF_LP_PARAMS


def _train_graph():
    g = gi.grid_deleted(24, 24, 0.15, 3)
    return g, 0.25


def test_training_lowers_the_oracle_loss_on_held_out_pairs():
    """Train on the GPU, then score the trained weights with the FP64 oracle on
    pairs the training never saw (other node, other right-hand sides)."""
    g, h = _train_graph()
    G, m = make(g, h)
    kappa, beta, k = 2.0, 0.75, 0.5
    G.precond_init(1)
    hist, npairs = G.precond_train(kappa, beta, k, epochs=30, seed=5)
    assert npairs > 1000
    assert np.all(np.isfinite(hist)) and hist[-1] < 0.7 * hist[0]
    w = learned.unflatten(G.precond_get().astype(np.float64))
    w0 = learned.init_params(1)
    t = 3.3  # between quadrature nodes
    inc, a, x = oracle_system(m, kappa, 1.0, t)
    S = dense_s_hat(inc, a)
    rng = np.random.default_rng(99)
    E = rng.standard_normal((4, inc.n_vertices))
    # smooth errors, the ones Jacobi-PCG leaves behind
    E = np.linalg.solve(S, np.linalg.solve(S, E.T)).T
    R = E @ S
    l_trained, _ = learned.loss_and_grad(w, inc, a, x, R, E)
    l_jacobi, _ = learned.loss_and_grad(w0, inc, a, x, R, E)
    assert l_trained < 0.8 * l_jacobi


@pytest.fixture(scope="module")
def trained():
    g, h = _train_graph()
    G, m = make(g, h)
    G.precond_init(1)
    G.precond_train(2.0, 0.75, 0.5, epochs=40, seed=5)
    return g, h, G, m


@pytest.mark.parametrize("layout", ["per_system", "staged"])
def test_learned_sample_matches_oracle(trained, layout):
    g, h, G, m = trained
    kappa, beta, k, seed, S = 2.0, 0.75, 0.5, 21, 5
    u, st = G.sample(kappa, beta, k, seed, S, precision="mixed", out_dtype="f64",
                     precond="learned", pcg_layout=layout)
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, h=h)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < 1e-4
    assert st["n_unconverged"] == 0 and st["numeric_flag"] == 0


def test_learned_preconditioner_needs_fewer_iterations_than_jacobi(trained):
    g, h, G, m = trained
    kappa, beta, k, seed, S = 2.0, 0.75, 0.5, 77, 8
    _, sj = G.sample(kappa, beta, k, seed, S, precision="mixed", precond="jacobi")
    _, sl = G.sample(kappa, beta, k, seed, S, precision="mixed", precond="learned")
    assert sl["n_precond_fallback"] == 0
    assert sl["pcg_iters_total"] < 0.8 * sj["pcg_iters_total"], (sl, sj)


def test_learned_path_in_graph_capture_and_integer_beta(trained):
    g, h, G, m = trained
    ml = fem.lumped_mass(m)
    out = torch.empty((3, G.n_dofs), dtype=torch.float64, device="cuda")
    for beta in (0.75, 1.25):
        d, _ = G.sample(2.0, beta, 0.5, 4, 3, precision="mixed", out_dtype="f64",
                        precond="learned")
        c, _ = G.sample(2.0, beta, 0.5, 4, 3, precision="mixed", out_dtype="f64",
                        precond="learned", out=out, use_graph=True)
        assert rel_l2(c.cpu().numpy(), d.cpu().numpy(), ml) < 1e-6
        _, ref, _ = sampler.sample(g, 2.0, beta, 0.5, 4, 3, h=h)
        assert rel_l2(c.cpu().numpy(), ref, ml) < 1e-4


@pytest.mark.parametrize("layout", ["per_system", "staged"])
def test_breakdown_falls_back_to_jacobi(layout):
    """exp(cs) underflows to 0 and N = 0: B = 0, r.z = 0 at the first step of
    every system, which must then finish with Jacobi and still match."""
    g, h = GRAPH()
    G, m = make(g, h)
    p = learned.init_params(0)
    p["cs"] = np.array(-200.0)
    G.precond_set(learned.flatten(p).astype(np.float32))
    kappa, beta, k, seed, S = 3.0, 0.6, 0.5, 8, 3
    u, st = G.sample(kappa, beta, k, seed, S, precision="mixed", out_dtype="f64",
                     precond="learned", pcg_layout=layout)
    assert st["n_precond_fallback"] == st["n_systems"]
    _, ref, _ = sampler.sample(g, kappa, beta, k, seed, S, h=h)
    assert rel_l2(u.cpu().numpy(), ref, fem.lumped_mass(m)) < 1e-4


def test_learned_option_errors():
    g, h = GRAPH()
    G, _ = make(g, h)
    with pytest.raises(grf.GrfError) as ei:  # no weights yet
        G.sample(2.0, 0.7, 0.5, 1, 2, precision="mixed", precond="learned")
    assert ei.value.code == grf.GRF_EINVAL
    G.precond_init(0)
    with pytest.raises(grf.GrfError) as ei:  # FP64 mode has no learned path
        G.sample(2.0, 0.7, 0.5, 1, 2, precision="fp64", precond="learned")
    assert ei.value.code == grf.GRF_ENOTSUP
    with pytest.raises(grf.GrfError):
        G.precond_set(np.zeros(10, np.float32))
    bad = np.zeros(grf.GRF_LP_PARAMS, np.float32)
    bad[3] = np.nan
    with pytest.raises(grf.GrfError):
        G.precond_set(bad)
