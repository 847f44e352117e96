"""FP64 reference of the learned BB^T preconditioner of the vertex Schur
systems. Test infrastructure only (see package header).

The paper's Phase 4 solves S^(l) u = g by PCG; the preconditioner here is
learned instead of Jacobi. Everything works on the Jacobi-scaled system
    S_hat = D^-1/2 S D^-1/2   (unit diagonal),
whose off-diagonal entry for an incidence k (vertex v, edge e to w) is
o_k = S^(e)_vw / sqrt(D_v D_w) <= 0; a_k = -o_k is the coupling weight.

Preconditioner: P = B B^T with B = diag(exp(s)) + N, N_vw = n_k on the
incidence pattern (B is not symmetric). P is symmetric positive definite when
B is nonsingular, and linear in the residual, so plain CG stays valid.

Network (weights shared by all nodes l and graphs):
    x_v = [1, log(1+deg)/3, sig, amax, sig^2, tanh(log t / 20), sig/deg, 0],
          sig = sum_k a_k, amax = max_k a_k over the incidences of v;
    h0 = relu(x W0 + b0);
    h_i = relu([h_{i-1}, m_i] W_i + b_i), m_i(v) = sum_k a_k h_{i-1}(nbr k), i = 1..3;
    s_v = h3_v . ws + cs;  n_k = a_k (h3_v . u + h3_w . up + cn)  (k: v -> w).
With the four heads at zero, B = I and P = I: exactly Jacobi on S.

Loss over pairs (r, e) with S_hat e = r:
    L = mean over pairs of (P r - e)^T S_hat (P r - e) / (r^T e),
the S_hat-energy norm of the preconditioned error relative to that of e.
"""
from __future__ import annotations

import numpy as np

F_IN = 8
H = 64
N_LAYERS = 3


def param_shapes():
    shapes = [("W0", (F_IN, H)), ("b0", (H,))]
    for i in range(1, N_LAYERS + 1):
        shapes += [(f"W{i}", (2 * H, H)), (f"b{i}", (H,))]
    shapes += [("ws", (H,)), ("cs", ()), ("u", (H,)), ("up", (H,)), ("cn", ())]
    return shapes


def n_params() -> int:
    return int(sum(int(np.prod(s)) for _, s in param_shapes()))


def unflatten(flat: np.ndarray) -> dict:
    p, off = {}, 0
    for name, shp in param_shapes():
        size = int(np.prod(shp))
        p[name] = flat[off:off + size].reshape(shp).astype(np.float64)
        off += size
    return p


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in param_shapes()])


class Incidence:
    """Vertex incidence lists of a graph (vertex v: edges e at v, other end w).
    dirs[k] = (edge, 0) when v is edge_u (entry B[u][v_e]), (edge, 1) otherwise."""

    def __init__(self, n_vertices, edge_u, edge_v):
        rows = [[] for _ in range(n_vertices)]
        for e, (a, b) in enumerate(zip(edge_u, edge_v)):
            rows[a].append((e, 0, b))
            rows[b].append((e, 1, a))
        self.vptr = np.zeros(n_vertices + 1, np.int64)
        self.vptr[1:] = np.cumsum([len(r) for r in rows])
        flat = [x for r in rows for x in r]
        self.edge = np.array([x[0] for x in flat], np.int64)
        self.side = np.array([x[1] for x in flat], np.int64)
        self.nbr = np.array([x[2] for x in flat], np.int64)
        self.src = np.repeat(np.arange(n_vertices), np.diff(self.vptr))
        self.n_vertices = n_vertices


def scaled_system(inc: Incidence, diag: np.ndarray, edge_off: np.ndarray):
    """a_k = -S^(e)_vw / sqrt(D_v D_w) per incidence."""
    return -edge_off[inc.edge] / np.sqrt(diag[inc.src] * diag[inc.nbr])


def features(inc: Incidence, a: np.ndarray, t: float) -> np.ndarray:
    V = inc.n_vertices
    deg = np.diff(inc.vptr).astype(np.float64)
    sig = np.zeros(V)
    np.add.at(sig, inc.src, a)
    amax = np.zeros(V)
    np.maximum.at(amax, inc.src, a)
    x = np.zeros((V, F_IN))
    x[:, 0] = 1.0
    x[:, 1] = np.log1p(deg) / 3.0
    x[:, 2] = sig
    x[:, 3] = amax
    x[:, 4] = sig * sig
    x[:, 5] = np.tanh(np.log(t) / 20.0)
    x[:, 6] = sig / np.maximum(deg, 1.0)
    return x


def _aggregate(inc: Incidence, a: np.ndarray, h: np.ndarray) -> np.ndarray:
    m = np.zeros_like(h)
    np.add.at(m, inc.src, a[:, None] * h[inc.nbr])
    return m


def forward(p: dict, inc: Incidence, a: np.ndarray, x: np.ndarray):
    """Returns s [V], n [2E] (incidence order) and the activations."""
    relu = lambda z: np.maximum(z, 0.0)
    hs = [relu(x @ p["W0"] + p["b0"])]
    ms = [None]
    for i in range(1, N_LAYERS + 1):
        m = _aggregate(inc, a, hs[-1])
        hs.append(relu(np.concatenate([hs[-1], m], axis=1) @ p[f"W{i}"] + p[f"b{i}"]))
        ms.append(m)
    h = hs[-1]
    s = h @ p["ws"] + p["cs"]
    alpha = h @ p["u"]
    beta = h @ p["up"]
    n = a * (alpha[inc.src] + beta[inc.nbr] + p["cn"])
    return s, n, (x, hs, ms, alpha, beta)


def b_apply_t(inc: Incidence, s, n, r):
    """y = B^T r: y_w = e^{s_w} r_w + sum over k (v -> w) n_k r_v."""
    y = np.exp(s) * r
    np.add.at(y, inc.nbr, n * r[inc.src])
    return y


def b_apply(inc: Incidence, s, n, y):
    """z = B y: z_v = e^{s_v} y_v + sum over k (v -> w) n_k y_w."""
    z = np.exp(s) * y
    np.add.at(z, inc.src, n * y[inc.nbr])
    return z


def precondition(inc, s, n, r):
    return b_apply(inc, s, n, b_apply_t(inc, s, n, r))


def s_hat_apply(inc: Incidence, a: np.ndarray, v: np.ndarray) -> np.ndarray:
    out = v.copy()
    np.add.at(out, inc.src, -a * v[inc.nbr])
    return out


def loss_and_grad(p: dict, inc: Incidence, a: np.ndarray, x: np.ndarray, R: np.ndarray,
                  E: np.ndarray, details: bool = False):
    """R, E: [P, V] pairs with S_hat e = r. Returns (loss, grads dict), and with
    details=True also the head gradients {"ds": dL/ds, "dn": dL/dn}."""
    s, n, (x, hs, ms, alpha, beta) = forward(p, inc, a, x)
    P = R.shape[0]
    ds = np.zeros_like(s)
    dn = np.zeros_like(n)
    loss = 0.0
    for r, e in zip(R, E):
        c = float(r @ e)
        y = b_apply_t(inc, s, n, r)
        z = b_apply(inc, s, n, y)
        eps = z - e
        q = s_hat_apply(inc, a, eps)
        loss += float(eps @ q) / c / P
        gz = 2.0 * q / c / P
        tt = b_apply_t(inc, s, n, gz)
        ds += np.exp(s) * (gz * y + r * tt)
        dn += gz[inc.src] * y[inc.nbr] + r[inc.src] * tt[inc.nbr]
    g = {}
    h = hs[-1]
    g["ws"] = h.T @ ds
    g["cs"] = np.array(ds.sum())
    dalpha = np.zeros(inc.n_vertices)
    dbeta = np.zeros(inc.n_vertices)
    np.add.at(dalpha, inc.src, a * dn)
    np.add.at(dbeta, inc.nbr, a * dn)
    g["cn"] = np.array((a * dn).sum())
    g["u"] = h.T @ dalpha
    g["up"] = h.T @ dbeta
    dh = ds[:, None] * p["ws"][None, :] + dalpha[:, None] * p["u"][None, :] + \
        dbeta[:, None] * p["up"][None, :]
    for i in range(N_LAYERS, 0, -1):
        da = dh * (hs[i] > 0)
        inp = np.concatenate([hs[i - 1], ms[i]], axis=1)
        g[f"W{i}"] = inp.T @ da
        g[f"b{i}"] = da.sum(axis=0)
        dinp = da @ p[f"W{i}"].T
        dh = dinp[:, :H] + _aggregate(inc, a, dinp[:, H:])
    da0 = dh * (hs[0] > 0)
    g["W0"] = x.T @ da0
    g["b0"] = da0.sum(axis=0)
    if details:
        return loss, g, {"ds": ds, "dn": dn}
    return loss, g


def init_params(seed: int) -> dict:
    """He-scaled random layers, zero heads (P = I at start)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in param_shapes():
        if name.startswith("W"):
            p[name] = rng.standard_normal(shp) * np.sqrt(2.0 / shp[0])
        else:
            p[name] = np.zeros(shp)
    return p
