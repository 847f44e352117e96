"""Lumped against consistent mass on the GPU (Sec. 4.3 performance comparison),
through the C ABI.

The graphs are the section's Barabasi-Albert family: attachment parameter m = 2,
unit edge lengths, h = 2^-6 on every edge (63 interior nodes per edge), from
100 up to 50 000 vertices. The section does not state kappa, beta or the
quadrature step; this harness takes the convergence study's kappa = 1 with
beta = 3/4 and its step k = -1/(beta ln h). Each graph is sampled twice with
the same launch knobs (sine-basis edge interiors on the tensor cores, the
library's PCG layout, one CUDA graph per call):
  lumped      W = M_L^{1/2} xi and M_L in the shifted operators (the method);
  consistent  W = R xi with M = R R^T, and M in the shifted operators.
For each it reports the first call's wall time (plans, and for the consistent
mass the host factorisation of the vertex mass Schur complement), the noise
phase alone (the section's "noise only" scenario) and the whole call (its
"full" scenario), both from CUDA events over several calls, and the device
memory the graph holds. The consistent mass is refused (GRF_ENOTSUP) where the
envelope of its vertex factor passes 2^27 entries; the row then says so.

    python -m paper_2605_02670_gb300.mass_comparison [n_vertices ...]
"""
from __future__ import annotations

import argparse
import json
import math
import statistics
import time

from . import GRF_ENOTSUP, Graph, GrfError

SIZES = (100, 500, 1000, 2000, 5000, 10000, 20000, 50000)


def ba_unit(n: int, seed: int = 0):
    import grf_inputs as gi
    return gi.barabasi_albert(n, 2, seed=seed, lengths="unit")


def time_mass(G: Graph, mass: str, kappa: float, beta: float, k: float, S: int, reps: int,
              flush) -> dict:
    import torch
    knobs = dict(precision="mixed", out_dtype="f32", interior="spectral_umma",
                 use_graph=True, mass=mass)
    out = torch.empty((S, G.n_dofs), dtype=torch.float32, device="cuda")
    free0 = torch.cuda.mem_get_info()[0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st = G.sample(kappa, beta, k, 1, S, out=out, timing=True, **knobs)
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    held = free0 - torch.cuda.mem_get_info()[0]
    stream = torch.cuda.current_stream()
    calls, noise = [], []
    for i in range(reps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, st = G.sample(kappa, beta, k, 2 + i, S, out=out, timing=True, **knobs)
        b.record(stream)
        b.synchronize()
        calls.append(a.elapsed_time(b))
        noise.append(st["phase_ms"]["noise"])
    ms = statistics.median(calls)
    return {"first_call_s": round(first_s, 4), "call_ms": ms, "noise_ms": statistics.median(noise),
            "samples_per_s": S / (ms / 1000.0), "pcg_iters_max": st["pcg_iters_max"],
            "device_bytes_held": int(held), "phase_ms": st["phase_ms"]}


def compare(n: int, S: int = 32, h: float = 2.0 ** -6, kappa: float = 1.0, beta: float = 0.75,
            reps: int = 5) -> dict:
    import torch
    g = ba_unit(n)
    k = -1.0 / (beta * math.log(h))
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device="cuda")  # 256 MB > L2
    row = {"n_vertices": n, "n_edges": int(len(g.edge_u)), "samples": S, "h": h, "kappa": kappa,
           "beta": beta, "k": k}
    for mass in ("lumped", "consistent"):
        G = Graph(g.edge_u, g.edge_v, g.lengths, g.n_vertices, h=h)
        row["n_dofs"] = G.n_dofs
        try:
            row[mass] = time_mass(G, mass, kappa, beta, k, S, reps, flush)
        except GrfError as err:
            if err.code != GRF_ENOTSUP:
                raise
            row[mass] = {"refused": str(err)}
        G.close()
        torch.cuda.empty_cache()
    if "call_ms" in row["consistent"]:
        row["consistent_over_lumped"] = {
            "full": row["consistent"]["call_ms"] / row["lumped"]["call_ms"],
            "noise": row["consistent"]["noise_ms"] / row["lumped"]["noise_ms"]}
    return row


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("sizes", nargs="*", type=int, default=list(SIZES))
    ap.add_argument("--samples", type=int, default=32)
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args(argv)
    for n in a.sizes:
        print(json.dumps(compare(n, S=a.samples, reps=a.reps)), flush=True)


if __name__ == "__main__":
    main()
