"""Python binding of the GB300 metric-graph Gaussian random field sampler.

Argument marshalling only: every step of the sampler runs in the CUDA kernels
of libgrf.so (built from csrc/ by build.py) behind the C ABI declared in
include/grf.h. PyTorch supplies device memory and streams. There is no CPU
path: if the library is missing, importing this package raises.

The functions carry the C names (grf_graph_create, grf_sample, ...); the
`Graph` class wraps a handle for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgrf.so")

GRF_OK, GRF_EINVAL, GRF_ENOMEM, GRF_ENOCONV, GRF_ECUDA, GRF_ENOTSUP, GRF_ENUMERIC = 0, -1, -2, -3, -4, -5, -6
GRF_FP64, GRF_MIXED = 0, 1
GRF_PRECOND_JACOBI, GRF_PRECOND_LEARNED, GRF_PRECOND_NEUMANN = 0, 1, 2
PRECONDS = {"jacobi": GRF_PRECOND_JACOBI, "learned": GRF_PRECOND_LEARNED,
            "neumann": GRF_PRECOND_NEUMANN}
GRF_LP_PARAMS = 25538
GRF_OUT_F64, GRF_OUT_F32 = 0, 1
GRF_PCG_AUTO, GRF_PCG_PER_SYSTEM, GRF_PCG_STAGED, GRF_PCG_STAGED_PAIRS, GRF_PCG_BATCHED = \
    0, 1, 2, 3, 4
PCG_LAYOUTS = {"auto": GRF_PCG_AUTO, "per_system": GRF_PCG_PER_SYSTEM, "staged": GRF_PCG_STAGED,
               "staged_pairs": GRF_PCG_STAGED_PAIRS, "batched": GRF_PCG_BATCHED}
GRF_INTERIOR_AUTO, GRF_INTERIOR_THOMAS, GRF_INTERIOR_SPECTRAL, GRF_INTERIOR_SPECTRAL_TC = 0, 1, 2, 3
GRF_INTERIOR_SPECTRAL_UMMA = 4
INTERIORS = {"auto": GRF_INTERIOR_AUTO, "thomas": GRF_INTERIOR_THOMAS,
             "spectral": GRF_INTERIOR_SPECTRAL, "spectral_tc": GRF_INTERIOR_SPECTRAL_TC, "spectral_umma": GRF_INTERIOR_SPECTRAL_UMMA}
GRF_SWEEP_AUTO, GRF_SWEEP_SEGMENTS, GRF_SWEEP_NODES = 0, 1, 2
SWEEPS = {"auto": GRF_SWEEP_AUTO, "segments": GRF_SWEEP_SEGMENTS, "nodes": GRF_SWEEP_NODES}
GRF_TIMING_ONLY = 1 << 30

C_SYMBOLS = ("grf_graph_create", "grf_graph_destroy", "grf_graph_info",
             "grf_graph_vertex_order", "grf_sample",
             "grf_sample_host", "grf_sample_host_stream", "grf_noise", "grf_apply", "grf_schur",
             "grf_vertex_solve",
             "grf_vertex_solve_noalloc", "grf_autotune", "grf_workspace_bytes",
             "grf_precond_init", "grf_precond_set", "grf_precond_get", "grf_precond_save",
             "grf_precond_load", "grf_precond_forward", "grf_precond_loss_grad",
             "grf_precond_train", "grf_last_error")


class GrfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"grf error {code}: {msg}")
        self.code = code


class grf_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("out_dtype", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("rtol", ctypes.c_double), ("timing", ctypes.c_int32),
                ("pcg_layout", ctypes.c_int32), ("recover_sg", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("interior", ctypes.c_int32),
                ("sweep", ctypes.c_int32), ("mass", ctypes.c_int32)]

    def knobs(self) -> dict:
        inv = {v: k for k, v in PCG_LAYOUTS.items()}
        inv_i = {v: k for k, v in INTERIORS.items()}
        inv_s = {v: k for k, v in SWEEPS.items()}
        return {"pcg_layout": inv[self.pcg_layout], "recover_sg": self.recover_sg,
                "interior": inv_i[self.interior], "sweep": inv_s[self.sweep]}


class grf_train_options(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("nodes_per_batch", ctypes.c_int32),
                ("n_samples", ctypes.c_int32), ("pairs_per_system", ctypes.c_int32),
                ("record_stride", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("rtol", ctypes.c_double), ("lr", ctypes.c_double), ("seed", ctypes.c_uint64)]


class grf_stats(ctypes.Structure):
    _fields_ = [("n_dofs", ctypes.c_int64), ("n_nodes", ctypes.c_int64),
                ("n_systems", ctypes.c_int64), ("pcg_iters_total", ctypes.c_int64),
                ("pcg_iters_max", ctypes.c_int32), ("n_unconverged", ctypes.c_int32),
                ("numeric_flag", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("n_precond_fallback", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("phase_ms", ctypes.c_double * 8)]

    PHASES = ("noise", "schur", "condense", "pcg", "recover", "layout", "precond_net", "unused")

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("phase_ms", "reserved")}
        d["phase_ms"] = dict(zip(self.PHASES, list(self.phase_ms)))
        return d


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2605_02670_gb300.build "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32, D, U64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64
    sig = {
        "grf_graph_create": [I64, I64, P, P, P, P, D, ctypes.POINTER(P)],
        "grf_graph_destroy": [P],
        "grf_graph_info": [P, P, P, P, P, P],
        "grf_graph_vertex_order": [P, P],
        "grf_sample": [P, D, D, D, U64, I64, P, P, P, P],
        "grf_sample_host": [P, D, D, D, U64, I64, P, P, P, P],
        "grf_sample_host_stream": [P, D, D, D, P, I64, I64, P, P, P, P],
        "grf_noise": [P, U64, I64, P, I32, P],
        "grf_apply": [P, D, I64, P, P, P, I64, P, P, P, P, P],
        "grf_schur": [P, D, D, D, P, P, P],
        "grf_vertex_solve": [P, D, D, D, I64, P, P, P, P, P, P],
        "grf_vertex_solve_noalloc": [P, D, D, D, I64, P, P, P, P, P, P],
        "grf_workspace_bytes": [P, D, D, I64, P, P],
        "grf_autotune": [P, D, D, D, I64, P, P, P, I32, P, P],
        "grf_precond_init": [P, U64],
        "grf_precond_set": [P, P, I64],
        "grf_precond_get": [P, P, I64],
        "grf_precond_save": [P, ctypes.c_char_p],
        "grf_precond_load": [P, ctypes.c_char_p],
        "grf_precond_forward": [P, D, D, D, P, P, P],
        "grf_precond_loss_grad": [P, D, D, D, I64, P, P, P, P, P],
        "grf_precond_train": [P, D, D, D, P, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.grf_last_error.argtypes = []
    lib.grf_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def _check(code: int, allow=(GRF_OK,)) -> int:
    if code not in allow:
        raise GrfError(code, _lib.grf_last_error().decode())
    return code


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def timing_flag(timing) -> int:
    """grf_options.timing from False/True (no phases / every phase) or an
    iterable of phase names (only those: GRF_TIMING_ONLY | their bits)."""
    if isinstance(timing, (bool, int)):
        return 1 if timing else 0
    names = list(timing)
    if not names:
        return 0
    return GRF_TIMING_ONLY | sum(1 << grf_stats.PHASES.index(n) for n in set(names))


GRF_MASS_LUMPED, GRF_MASS_CONSISTENT = 0, 1
MASSES = {"lumped": GRF_MASS_LUMPED, "consistent": GRF_MASS_CONSISTENT}


def make_options(precision="fp64", out_dtype=None, rtol=0.0, max_iter=0,
                 timing=False, pcg_layout="auto", recover_sg=0, use_graph=False,
                 precond="jacobi", interior="auto", sweep="auto", mass="lumped") -> grf_options:
    """timing: False, True (every phase) or phase names to time only those."""
    prec = {"fp64": GRF_FP64, "mixed": GRF_MIXED}[precision]
    if out_dtype is None:
        out_dtype = "f64" if prec == GRF_FP64 else "f32"
    od = {"f64": GRF_OUT_F64, "f32": GRF_OUT_F32}[out_dtype]
    return grf_options(prec, PRECONDS[precond], od, int(max_iter), float(rtol),
                       timing_flag(timing), PCG_LAYOUTS[pcg_layout], int(recover_sg),
                       1 if use_graph else 0, INTERIORS[interior], SWEEPS[sweep], MASSES[mass])


# ------------------------------------------------------------ C-named functions


def grf_graph_create(edge_u, edge_v, lengths, n_vertices: int, h: float | None = None,
                     n_elems=None) -> ctypes.c_void_p:
    eu = np.ascontiguousarray(edge_u, dtype=np.int64)
    ev = np.ascontiguousarray(edge_v, dtype=np.int64)
    ln = np.ascontiguousarray(lengths, dtype=np.float64)
    ne_ptr = None
    if n_elems is not None:
        ne = np.ascontiguousarray(n_elems, dtype=np.int32)
        ne_ptr = _ptr(ne)
    handle = ctypes.c_void_p()
    _check(_lib.grf_graph_create(int(n_vertices), int(eu.shape[0]), _ptr(eu), _ptr(ev), _ptr(ln),
                                 ne_ptr, float(h) if h is not None else 0.0, ctypes.byref(handle)))
    return handle


def grf_graph_destroy(handle) -> None:
    _check(_lib.grf_graph_destroy(handle))


def grf_graph_info(handle, n_vertices_in: int, n_edges: int) -> dict:
    n, nk, ni = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    vmap = np.empty(n_vertices_in, np.int64)
    offs = np.empty(n_edges + 1, np.int64)
    _check(_lib.grf_graph_info(handle, ctypes.byref(n), ctypes.byref(nk), ctypes.byref(ni),
                               _ptr(vmap), _ptr(offs)))
    return {"n_dofs": n.value, "n_kept_vertices": nk.value, "n_interior": ni.value,
            "vertex_map": vmap, "interior_offsets": offs}


def grf_graph_vertex_order(handle, n_kept: int) -> np.ndarray:
    perm = np.empty(n_kept, np.int64)
    _check(_lib.grf_graph_vertex_order(handle, _ptr(perm)))
    return perm


def grf_sample(handle, kappa, beta, k_step, seed, n_samples, out_ptr: int, opts: grf_options,
               stream=None, allow_noconv=False) -> dict:
    st = grf_stats()
    allow = (GRF_OK, GRF_ENOCONV) if allow_noconv else (GRF_OK,)
    _check(_lib.grf_sample(handle, float(kappa), float(beta), float(k_step), int(seed),
                           int(n_samples), ctypes.c_void_p(out_ptr), ctypes.byref(opts),
                           _stream(stream), ctypes.byref(st)), allow)
    return st.as_dict()


def grf_sample_host(handle, kappa, beta, k_step, seed, n_samples, out: np.ndarray,
                    opts: grf_options, stream=None) -> dict:
    st = grf_stats()
    _check(_lib.grf_sample_host(handle, float(kappa), float(beta), float(k_step), int(seed),
                                int(n_samples), _ptr(out), ctypes.byref(opts), _stream(stream),
                                ctypes.byref(st)))
    return st.as_dict()


def grf_sample_host_stream(handle, kappa, beta, k_step, seeds, n_samples, outs,
                           opts: grf_options, stream=None) -> dict:
    """len(seeds) pipelined host draws into the host arrays outs (one per seed)."""
    sd = np.ascontiguousarray(seeds, np.uint64)
    ptrs = (ctypes.c_void_p * len(outs))(*[o.ctypes.data for o in outs])
    st = grf_stats()
    _check(_lib.grf_sample_host_stream(handle, float(kappa), float(beta), float(k_step),
                                       _ptr(sd), int(sd.shape[0]), int(n_samples), ptrs,
                                       ctypes.byref(opts), _stream(stream), ctypes.byref(st)))
    return st.as_dict()


def grf_noise(handle, seed, n_samples, out_ptr: int, raw_words, stream=None) -> None:
    """raw_words: 0 (or False) lumped noise in FP64, 1 (or True) the uint32
    words, 2 the consistent-mass noise in FP64."""
    _check(_lib.grf_noise(handle, int(seed), int(n_samples), ctypes.c_void_p(out_ptr),
                          int(raw_words), _stream(stream)))


def grf_apply(handle, kappa, alpha, gamma, weight, n_rhs, rhs_ptr: int, out_ptr: int,
              opts: grf_options, stream=None) -> dict:
    a = np.ascontiguousarray(alpha, np.float64)
    g = np.ascontiguousarray(gamma, np.float64)
    w = np.ascontiguousarray(weight, np.float64)
    st = grf_stats()
    _check(_lib.grf_apply(handle, float(kappa), int(a.shape[0]), _ptr(a), _ptr(g), _ptr(w),
                          int(n_rhs), ctypes.c_void_p(rhs_ptr), ctypes.c_void_p(out_ptr),
                          ctypes.byref(opts), _stream(stream), ctypes.byref(st)))
    return st.as_dict()


def grf_schur(handle, kappa, alpha, gamma, diag_ptr: int, off_ptr: int, stream=None) -> None:
    _check(_lib.grf_schur(handle, float(kappa), float(alpha), float(gamma),
                          ctypes.c_void_p(diag_ptr), ctypes.c_void_p(off_ptr), _stream(stream)))


def grf_vertex_solve(handle, kappa, alpha, gamma, n_rhs, rhs_ptr: int, g_ptr: int, u_ptr: int,
                     opts: grf_options, stream=None) -> dict:
    st = grf_stats()
    _check(_lib.grf_vertex_solve(handle, float(kappa), float(alpha), float(gamma), int(n_rhs),
                                 ctypes.c_void_p(rhs_ptr), ctypes.c_void_p(g_ptr),
                                 ctypes.c_void_p(u_ptr), ctypes.byref(opts), _stream(stream),
                                 ctypes.byref(st)))
    return st.as_dict()


def grf_vertex_solve_noalloc(handle, kappa, alpha, gamma, n_rhs, rhs_ptr: int, g_ptr: int,
                             u_ptr: int, opts: grf_options, stream=None) -> dict:
    """grf_vertex_solve for callers that cannot allocate device memory: its
    scratch is a fixed 16 MiB static device array inside the library. The
    graph must already have been used on this device by an allocating call;
    concurrent calls on the GPU race on the shared array."""
    st = grf_stats()
    _check(_lib.grf_vertex_solve_noalloc(handle, float(kappa), float(alpha), float(gamma),
                                         int(n_rhs), ctypes.c_void_p(rhs_ptr),
                                         ctypes.c_void_p(g_ptr), ctypes.c_void_p(u_ptr),
                                         ctypes.byref(opts), _stream(stream), ctypes.byref(st)))
    return st.as_dict()


def grf_autotune(handle, kappa, beta, k_step, n_samples, out_ptr: int, base: grf_options,
                 stream=None, reps=2):
    """Fastest launch knobs for this configuration; returns (options, ms)."""
    best = grf_options()
    ms = ctypes.c_double()
    _check(_lib.grf_autotune(handle, float(kappa), float(beta), float(k_step), int(n_samples),
                             ctypes.c_void_p(out_ptr), ctypes.byref(base), _stream(stream),
                             int(reps), ctypes.byref(best), ctypes.byref(ms)))
    return best, ms.value


def grf_workspace_bytes(handle, beta, k_step, n_samples, opts: grf_options) -> int:
    b = ctypes.c_size_t()
    _check(_lib.grf_workspace_bytes(handle, float(beta), float(k_step), int(n_samples),
                                    ctypes.byref(opts), ctypes.byref(b)))
    return b.value


def grf_precond_init(handle, seed: int) -> None:
    _check(_lib.grf_precond_init(handle, int(seed)))


def grf_precond_set(handle, params) -> None:
    p = np.ascontiguousarray(params, np.float32)
    _check(_lib.grf_precond_set(handle, _ptr(p), int(p.size)))


def grf_precond_get(handle) -> np.ndarray:
    p = np.empty(GRF_LP_PARAMS, np.float32)
    _check(_lib.grf_precond_get(handle, _ptr(p), int(p.size)))
    return p


def grf_precond_save(handle, path: str) -> None:
    _check(_lib.grf_precond_save(handle, os.fsencode(path)))


def grf_precond_load(handle, path: str) -> None:
    _check(_lib.grf_precond_load(handle, os.fsencode(path)))


def grf_precond_forward(handle, kappa, alpha, gamma, n_kept: int, n_edges: int, stream=None):
    """Network output (s [n_kept], n [2 n_edges]) for A = alpha M_L + gamma K."""
    s = np.empty(n_kept, np.float32)
    n = np.empty(2 * n_edges, np.float32)
    _check(_lib.grf_precond_forward(handle, float(kappa), float(alpha), float(gamma), _ptr(s),
                                    _ptr(n), _stream(stream)))
    return s, n


def grf_precond_loss_grad(handle, kappa, alpha, gamma, R, E, stream=None):
    """Loss and FP32 gradient over host pairs R, E [n_pairs][n_kept]."""
    R = np.ascontiguousarray(R, np.float32)
    E = np.ascontiguousarray(E, np.float32)
    assert R.shape == E.shape and R.ndim == 2
    loss = ctypes.c_double()
    grad = np.empty(GRF_LP_PARAMS, np.float32)
    _check(_lib.grf_precond_loss_grad(handle, float(kappa), float(alpha), float(gamma),
                                      int(R.shape[0]), _ptr(R), _ptr(E), ctypes.byref(loss),
                                      _ptr(grad), _stream(stream)))
    return loss.value, grad


def grf_precond_train(handle, kappa, beta, k_step, opts: grf_train_options, stream=None):
    """Trains the handle's network; returns (per-epoch mean loss, pairs recorded)."""
    hist = np.zeros(max(int(opts.epochs), 1) if opts.epochs > 0 else 40, np.float32)
    npairs = ctypes.c_int64()
    _check(_lib.grf_precond_train(handle, float(kappa), float(beta), float(k_step),
                                  ctypes.byref(opts), _ptr(hist), ctypes.byref(npairs),
                                  _stream(stream)))
    return hist, npairs.value


# ------------------------------------------------------------ convenience wrapper


class Graph:
    """A metric graph handle with torch-tensor helpers (device memory only)."""

    def __init__(self, edge_u, edge_v, lengths, n_vertices: int, h: float | None = None,
                 n_elems=None):
        self.n_vertices_in = int(n_vertices)
        self.n_edges = int(np.asarray(edge_u).shape[0])
        self.edge_u_in = np.asarray(edge_u, np.int64).copy()
        self.edge_v_in = np.asarray(edge_v, np.int64).copy()
        self.handle = grf_graph_create(edge_u, edge_v, lengths, n_vertices, h, n_elems)
        info = grf_graph_info(self.handle, self.n_vertices_in, self.n_edges)
        self.n_dofs = info["n_dofs"]
        self.n_kept = info["n_kept_vertices"]
        self.n_interior = info["n_interior"]
        self.vertex_map = info["vertex_map"]
        self.interior_offsets = info["interior_offsets"]

    @property
    def vertex_order(self) -> np.ndarray:
        """Slot -> kept vertex id of the sample-group PCG's shared-memory layout."""
        return grf_graph_vertex_order(self.handle, self.n_kept)

    def close(self):
        if getattr(self, "handle", None) is not None:
            grf_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sample(self, kappa, beta, k_step, seed, n_samples, precision="fp64", out_dtype=None,
               rtol=0.0, max_iter=0, out=None, stream=None, allow_noconv=False, timing=False,
               pcg_layout="auto", recover_sg=0, use_graph=False, precond="jacobi",
               interior="auto", sweep="auto", mass="lumped"):
        import torch
        opts = make_options(precision, out_dtype, rtol, max_iter, timing, pcg_layout, recover_sg,
                            use_graph, precond, interior, sweep, mass)
        dt = torch.float64 if opts.out_dtype == GRF_OUT_F64 else torch.float32
        if out is None:
            out = torch.empty((n_samples, self.n_dofs), dtype=dt, device="cuda")
        assert out.dtype == dt and out.is_cuda and out.is_contiguous()
        assert tuple(out.shape) == (n_samples, self.n_dofs)
        stats = grf_sample(self.handle, kappa, beta, k_step, seed, n_samples, out.data_ptr(),
                           opts, stream, allow_noconv)
        return out, stats

    def sample_host(self, kappa, beta, k_step, seed, n_samples, precision="fp64",
                    out_dtype=None, rtol=0.0, max_iter=0, out=None, stream=None, timing=False,
                    precond="jacobi", pcg_layout="auto", recover_sg=0, interior="auto",
                    use_graph=False, sweep="auto", mass="lumped"):
        opts = make_options(precision, out_dtype, rtol, max_iter, timing, pcg_layout, recover_sg,
                            use_graph, precond=precond, interior=interior, sweep=sweep, mass=mass)
        dt = np.float64 if opts.out_dtype == GRF_OUT_F64 else np.float32
        if out is None:
            out = np.empty((n_samples, self.n_dofs), dtype=dt)
        stats = grf_sample_host(self.handle, kappa, beta, k_step, seed, n_samples, out, opts,
                                stream)
        return out, stats

    def sample_host_stream(self, kappa, beta, k_step, seeds, n_samples, precision="fp64",
                           out_dtype=None, outs=None, stream=None, **knobs):
        """One host array per seed, drawn back to back with the host copies of
        one call overlapping the next call's compute."""
        opts = make_options(precision, out_dtype, **knobs)
        dt = np.float64 if opts.out_dtype == GRF_OUT_F64 else np.float32
        if outs is None:
            outs = [np.empty((n_samples, self.n_dofs), dtype=dt) for _ in seeds]
        stats = grf_sample_host_stream(self.handle, kappa, beta, k_step, seeds, n_samples, outs,
                                       opts, stream)
        return outs, stats

    def autotune(self, kappa, beta, k_step, n_samples, precision="fp64", out_dtype=None,
                 rtol=0.0, max_iter=0, reps=2, stream=None, precond="jacobi"):
        """Times the launch knobs and returns ({pcg_layout, recover_sg}, ms per call)."""
        import torch
        base = make_options(precision, out_dtype, rtol, max_iter, precond=precond)
        dt = torch.float64 if base.out_dtype == GRF_OUT_F64 else torch.float32
        out = torch.empty((n_samples, self.n_dofs), dtype=dt, device="cuda")
        best, ms = grf_autotune(self.handle, kappa, beta, k_step, n_samples, out.data_ptr(), base,
                                stream, reps)
        return best.knobs(), ms

    def noise(self, seed, n_samples, raw=False, stream=None, mass="lumped"):
        """raw: the uint32 Philox words; mass="consistent": W = R xi of the
        consistent mass (FP64 output of the FP32 computation)."""
        import torch
        dt = torch.int32 if raw else torch.float64
        out = torch.empty((n_samples, self.n_dofs), dtype=dt, device="cuda")
        grf_noise(self.handle, seed, n_samples, out.data_ptr(),
                  2 if mass == "consistent" else (1 if raw else 0), stream)
        return out

    def apply(self, kappa, alpha, gamma, weight, rhs, precision="fp64", out_dtype=None,
              rtol=0.0, max_iter=0, stream=None, interior="auto", sweep="auto", mass="lumped"):
        import torch
        opts = make_options(precision, out_dtype, rtol, max_iter, interior=interior, sweep=sweep,
                            mass=mass)
        rhs = rhs.to(dtype=torch.float64).contiguous()
        dt = torch.float64 if opts.out_dtype == GRF_OUT_F64 else torch.float32
        out = torch.empty(tuple(rhs.shape), dtype=dt, device="cuda")
        stats = grf_apply(self.handle, kappa, alpha, gamma, weight, rhs.shape[0], rhs.data_ptr(),
                          out.data_ptr(), opts, stream)
        return out, stats

    def schur(self, kappa, alpha, gamma, stream=None):
        import torch
        diag = torch.empty(self.n_kept, dtype=torch.float64, device="cuda")
        off = torch.empty(self.n_edges, dtype=torch.float64, device="cuda")
        grf_schur(self.handle, kappa, alpha, gamma, diag.data_ptr(), off.data_ptr(), stream)
        return diag, off

    def vertex_solve(self, kappa, alpha, gamma, rhs, precision="fp64", rtol=0.0, max_iter=0,
                     stream=None, precond="jacobi", interior="auto"):
        import torch
        opts = make_options(precision, None, rtol, max_iter, precond=precond, interior=interior)
        rhs = rhs.to(dtype=torch.float64).contiguous()
        g = torch.empty((rhs.shape[0], self.n_kept), dtype=torch.float64, device="cuda")
        u = torch.empty_like(g)
        stats = grf_vertex_solve(self.handle, kappa, alpha, gamma, rhs.shape[0], rhs.data_ptr(),
                                 g.data_ptr(), u.data_ptr(), opts, stream)
        return g, u, stats

    def workspace_bytes(self, beta, k_step, n_samples, precision="fp64", precond="jacobi") -> int:
        return grf_workspace_bytes(self.handle, beta, k_step, n_samples,
                                   make_options(precision, precond=precond))

    # learned B B^T preconditioner of the vertex systems
    def precond_init(self, seed=0):
        grf_precond_init(self.handle, seed)

    def precond_set(self, params):
        grf_precond_set(self.handle, params)

    def precond_get(self) -> np.ndarray:
        return grf_precond_get(self.handle)

    def precond_save(self, path):
        grf_precond_save(self.handle, path)

    def precond_load(self, path):
        grf_precond_load(self.handle, path)

    def precond_forward(self, kappa, alpha, gamma, stream=None):
        return grf_precond_forward(self.handle, kappa, alpha, gamma, self.n_kept, self.n_edges,
                                   stream)

    def precond_loss_grad(self, kappa, alpha, gamma, R, E, stream=None):
        return grf_precond_loss_grad(self.handle, kappa, alpha, gamma, R, E, stream)

    def precond_train(self, kappa, beta, k_step, epochs=40, nodes_per_batch=8, n_samples=8,
                      pairs_per_system=16, record_stride=2, max_iter=0, rtol=0.0, lr=1e-3,
                      seed=0, stream=None):
        o = grf_train_options(int(epochs), int(nodes_per_batch), int(n_samples),
                              int(pairs_per_system), int(record_stride), int(max_iter),
                              float(rtol), float(lr), int(seed))
        return grf_precond_train(self.handle, kappa, beta, k_step, o, stream)


def mesh_elements(lengths, h: float, clip=None) -> np.ndarray:
    """Per-edge element counts n_e = ceil(l_e / h) (Sec. 3, Phase 1), optionally
    clipped to [lo, hi], as int32 for grf_graph_create."""
    n = np.ceil(np.asarray(lengths, np.float64) / h)
    if clip is not None:
        n = np.clip(n, clip[0], clip[1])
    return np.maximum(n, 1).astype(np.int32)
