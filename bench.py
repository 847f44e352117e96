#!/usr/bin/env python
"""Throughput of the metric-graph Gaussian random field sampler on GB300.

One step = one grf_sample call: noise, per-node Schur blocks, condensed
right-hand sides, vertex PCG, fused interior recovery + quadrature sum, for
every quadrature node and every sample of the workload. Default workload: the
2000-vertex random geometric graph (~5000 edges, h = 2^-10, kappa = 10,
beta = 0.75, k = 0.3, 16 samples, FP32 edge sweeps with FP64 Schur/PCG/sum).

Prints one JSON line. --impl reference times the FP64 CPU oracle instead.
With torchrun (N > 1) every rank draws its own samples (independent
replicas, seed offset by rank): weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import grf_inputs as gi  # noqa: E402

METRIC = "field samples/s and DOF-solves/s at rel L2 ≤1e-4 vs FP64 oracle; HBM % of peak"
UNIT = "samples/s"
# L2 size used by the CPU-side work model when no device is there to ask
L2_BYTES = 129 * 1024 * 1024


def quad_count(beta, k):
    f = beta - math.floor(beta)
    km = math.ceil(math.pi ** 2 / (4 * k * k * f))
    kp = math.ceil(math.pi ** 2 / (4 * k * k * (1 - f)))
    return km + kp + 1


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["hbm_gbs"], "measured"
    return 6800.0, "fallback"


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a rank's replica: ranks draw disjoint sample streams (the noise
    counter runs over (DOF, sample) under a per-seed key)."""
    return seed + 1000003 * rank


def max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest of the ranks' values (the job ends with its slowest rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / seconds


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def traffic_record(kernel_file: str, workload: str):
    """dram bytes per launch from a committed ncu summary, valid only while the
    kernel source is unchanged (its sha256 is stored beside the figure)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(f"{kernel_file}:{workload}")
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2605_02670_gb300", "csrc", kernel_file)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return rec["bytes_per_launch"] if rec.get("sha256") == h else None


# ----------------------------------------------------------------- CPU oracle

# Above this many DOFs the oracle is timed on a smaller graph of the same family
# (same parameters, edge statistics and mesh size) and its cost scaled by the
# DOF ratio: one sparse LU of the 78 M-DOF lattice takes minutes.
ORACLE_MAX_DOFS = 2_000_000
ORACLE_SUBGRAPHS = {"grid": {"nx": 20, "ny": 20}, "ba": {"n": 1000}}


def oracle_graph(w, graph):
    """(graph, mesh of it, scale): the graph the oracle is timed on and the
    factor N_workload / N_timed that takes its cost to the workload."""
    from oracle import fem
    mesh = _oracle_mesh(w, graph)
    if mesh.n_dofs <= ORACLE_MAX_DOFS or w.graph_args["kind"] not in ORACLE_SUBGRAPHS:
        return graph, mesh, 1.0
    args = dict(w.graph_args)
    args.update(ORACLE_SUBGRAPHS[args["kind"]])
    kind = args.pop("kind")
    sub = {"grid": gi.grid_deleted, "ba": gi.barabasi_albert}[kind](**args)
    sm = _oracle_mesh(w, sub)
    return sub, sm, mesh.n_dofs / sm.n_dofs


def _oracle_mesh(w, graph):
    from oracle import fem
    ne = np.clip(np.ceil(graph.lengths / w.h), *w.clip) if w.clip else None
    return fem.build_mesh(graph.edge_u, graph.edge_v, graph.lengths, graph.n_vertices, h=w.h,
                          n_elems=ne)


def _oracle_nodes(wdict, graph, node_ids):
    """One worker's share: assembly and noise, then the listed quadrature
    nodes (each one sparse LU and S solves). Returns (fixed s, per-node s)."""
    import math as _m

    from oracle import fem, noise, quadrature, sampler
    t0 = time.perf_counter()
    ne = np.clip(np.ceil(graph.lengths / wdict["h"]), *wdict["clip"]) if wdict["clip"] else None
    mesh = fem.build_mesh(graph.edge_u, graph.edge_v, graph.lengths, graph.n_vertices,
                          h=wdict["h"], n_elems=ne)
    ml, _, kmat = sampler.assemble(mesh, wdict["kappa"])
    b = noise.white_noise(ml, wdict["seed"], wdict["n_samples"])
    t_fixed = time.perf_counter() - t0
    f = wdict["beta"] - _m.floor(wdict["beta"])
    t, wt = quadrature.nodes(f, wdict["k_step"])
    t1 = time.perf_counter()
    for i in node_ids:
        sampler.shifted_sum(ml, kmat, b, [t[i]], [wt[i]])
    return t_fixed, (time.perf_counter() - t1) / max(1, len(node_ids))


def _wdict(w):
    return {"h": w.h, "clip": w.clip, "kappa": w.kappa, "beta": w.beta, "k_step": w.k_step,
            "seed": w.seed, "n_samples": w.n_samples}


def oracle_sample(w, graph, n_nodes_sample=32, parallel=False):
    """Time the FP64 oracle on a bounded sample of the workload: mesh, assembly
    and noise for all samples, then `n_nodes_sample` of the L quadrature nodes
    (spread over the range), each factorised once and solved for every sample;
    extrapolated linearly in the node count (and by the DOF ratio when a
    smaller graph of the family stands in). parallel: the paper's
    parallelisation, every quadrature node, dealt round-robin over every host
    core (one process each, started with spawn), each core after its own
    assembly; the time is the slowest core's (only the DOF ratio is
    extrapolated)."""
    g, mesh, scale = oracle_graph(w, graph)
    # beta >= 1: one more factorisation per integer power, timed like a node
    Lq = quad_count(w.beta, w.k_step)
    L = Lq + int(math.floor(w.beta))
    t0 = time.perf_counter()
    if not parallel:
        pick = np.linspace(0, Lq - 1, n_nodes_sample).round().astype(int).tolist()
        t_fixed, t_node = _oracle_nodes(_wdict(w), g, pick)
        cores = 1
        total = (t_fixed + t_node * L) * scale
        how = f"{len(pick)} of {L} quadrature nodes, single thread"
    else:
        import concurrent.futures as cf
        import multiprocessing as mp
        cores = min(os.cpu_count() or 1, Lq)
        shares = [list(range(c, Lq, cores)) for c in range(cores)]
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        # a worker that dies raises BrokenProcessPool here instead of hanging
        with cf.ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn")) as ex:
            futs = [ex.submit(_oracle_nodes, _wdict(w), g, ids) for ids in shares]
            res = [f.result(timeout=900) for f in futs]
        per_core = [r[0] + r[1] * len(ids) for r, ids in zip(res, shares)]
        # beta >= 1: the integer powers run after the sum, one solve each
        t_node = max(r[1] for r in res)
        total = (max(per_core) + t_node * (L - Lq)) * scale
        how = (f"all {Lq} quadrature nodes dealt round-robin over {cores} cores (spawned "
               f"processes; the slowest core's time)")
    wall = time.perf_counter() - t0
    where = (f"{w.name}" if scale == 1.0 else
             f"a {mesh.n_dofs}-DOF graph of the {w.name} family (same parameters and mesh "
             f"size), scaled by the DOF ratio {scale:.1f}")
    return {"value": w.n_samples / total, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"{where}: mesh+assembly+noise for {w.n_samples} samples, then {how} "
                       f"(SuperLU factorisation + {w.n_samples} solves each)"
                       + ("" if parallel else f", extrapolated linearly to all {L} nodes")
                       + f"; measured {wall:.1f} s"),
            "wall_s": wall}


def run_reference(args, w, graph):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # the oracle keeps no state between calls, so it needs no warm-up;
    # every step is one timed bounded sample
    vals, walls = [], []
    cb = None
    for _ in range(args.steps):
        cb = oracle_sample(w, graph, parallel=True)
        vals.append(cb["value"])
        walls.append(cb.pop("wall_s"))
    v = statistics.median(vals)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.mean(walls),
            "ms_per_step_is": "wall time of one bounded oracle sample (cpu_baseline.sample); "
                              "value is that sample extrapolated to the whole workload",
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name}, "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU path


def algorithmic(w, G, stats, phase, S, tsize, out_size, l2_bytes=L2_BYTES):
    """Algorithmic bytes (or flops) of one launch of a phase, from the
    method's per-unit figures (b = bytes per value of the phase's arithmetic:
    4 in mixed precision, 8 in FP64):
    noise: writes N S b and reads the N mass factors (b bytes each);
    PCG, per system-iteration: 4 (|V| + 2|E|) + 10 |V| flops; when the vertex
    vectors of all systems exceed L2, 10 |V| b bytes of vector traffic plus the
    node's matrix, (|V| + |E|) (8 + 4) bytes, shared over the S samples;
    condensation + recovery: 12 flops per (interior node, node, sample),
    4 of them in the two end sweeps of the condensation and 8 in the recovery
    (forward/back sweep and the weighted accumulation);
    Schur blocks: the FP64 words written per node."""
    N, V, E, NI = G.n_dofs, G.n_kept, G.n_edges, G.n_interior
    L = stats["n_nodes"]
    if phase == "noise":
        return N * S * tsize + N * tsize, "hbm"
    if phase == "pcg":
        it = stats["pcg_iters_total"]
        if L * S * V * 8 <= l2_bytes:
            return it * (4 * (V + 2 * E) + 10 * V), "alu"
        return it * 10 * V * tsize + (it / S) * (V + E) * 12, "hbm"
    if phase == "recover":
        return 8.0 * NI * L * S, "alu"
    if phase == "condense":
        return 4.0 * NI * L * S, "alu"
    if phase == "schur":
        return L * (E * 16 + V * 8 + 2 * E * 8), "hbm"
    return 0, "hbm"


def fp32_peak_tflops(sm_mhz, n_sm=152):
    # SMs x 128 FP32 lanes x 2 flops (FMA) per clock
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


# Same family and parameters, small enough for the oracle to solve every node
# in seconds: the accuracy of the bench's configuration against the oracle.
CHECK_GRAPHS = {
    "grid": lambda a: gi.grid_deleted(6, 6, a.get("frac", 0.15), seed=a.get("seed", 7)),
    "rgg": lambda a: gi.random_geometric(300, a.get("radius", 0.0285) * math.sqrt(2000 / 300),
                                         seed=a.get("seed", 0)),
    "ba": lambda a: gi.barabasi_albert(80, a.get("m", 3), seed=a.get("seed", 0)),
    "long": lambda a: gi.long_edges(20, 20, a.get("n_elems", 3072), a.get("spread", 64),
                                    a.get("h", 2.0 ** -9), seed=a.get("seed", 0)),
}


def ml_weights(graph, ne, G):
    """Lumped-mass diagonal in the library's DOF order ([kept vertices], then
    the interior nodes edge by edge): h_e on an edge's interior nodes, the sum
    of h_e / 2 over the incident edges on a vertex."""
    he = np.asarray(graph.lengths, np.float64) / ne
    vm = np.asarray(G.vertex_map)
    wv = np.zeros(G.n_kept)
    np.add.at(wv, vm[np.asarray(graph.edge_u)], he / 2)
    np.add.at(wv, vm[np.asarray(graph.edge_v)], he / 2)
    return np.concatenate([wv, np.repeat(he, np.asarray(ne, np.int64) - 1)])


def accuracy_checks(args, w, graph, G, out, seed, prec, knobs):
    """GPU side of the accuracy figures of the benchmarked configuration:
    (1) the same parameters, mesh size and launch knobs on a small graph of
    the workload's family (4 samples), kept for the CPU leg's oracle;
    (2) at full size, the last timed call's first two samples against the
    plain FP64 form on the same GPU (same seed), whose rate is timed too."""
    import torch
    import paper_2605_02670_gb300 as grf

    res = {}
    kind = w.graph_args["kind"]
    cg = CHECK_GRAPHS[kind](w.graph_args) if kind in CHECK_GRAPHS else graph
    ne = grf.mesh_elements(cg.lengths, w.h, w.clip)
    Gc = grf.Graph(cg.edge_u, cg.edge_v, cg.lengths, cg.n_vertices, n_elems=ne)
    Sc = min(4, w.n_samples)
    uc, _ = Gc.sample(w.kappa, w.beta, w.k_step, w.seed, Sc, precision=prec, out_dtype="f64",
                      use_graph=args.use_graph, **knobs)
    mass = knobs.get("mass", "lumped")
    res["_check"] = (cg, ne, Sc, uc.cpu().numpy(), Gc.n_dofs, mass)
    if prec == "mixed" and mass == "lumped":
        S2 = 2
        u64, _ = G.sample(w.kappa, w.beta, w.k_step, seed, S2, precision="fp64")
        mlf = ml_weights(graph, grf.mesh_elements(graph.lengths, w.h, w.clip), G)
        res["full_vs_fp64_form"] = {
            "rel_l2": _rel_l2(out[:S2].double().cpu().numpy(), u64.cpu().numpy(), mlf),
            "samples": S2}
        del u64
        # the plain FP64 form (FP64 Thomas interiors, FP64 Jacobi-PCG), timed
        st = torch.cuda.current_stream()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        G.sample(w.kappa, w.beta, w.k_step, seed + 1, S2, precision="fp64")
        b.record(st)
        b.synchronize()
        res["fp64_form"] = {"value": S2 / (a.elapsed_time(b) / 1000.0), "unit": UNIT,
                            "samples_per_call": S2}
        torch.cuda.empty_cache()
    return res


def oracle_check(w, check):
    """CPU leg: the oracle's field on the small check graph and the relative
    M_L-weighted L2 error of the GPU's field there."""
    from oracle import consistent, fem, sampler
    cg, ne, Sc, uc, n, mass = check
    if mass == "consistent":
        m, ref, _ = consistent.sample(cg, w.kappa, w.beta, w.k_step, w.seed, Sc, n_elems=ne)
    else:
        m, ref, _ = sampler.sample(cg, w.kappa, w.beta, w.k_step, w.seed, Sc, n_elems=ne)
    return {"rel_l2": _rel_l2(uc, ref, fem.lumped_mass(m)), "mass": mass,
            "graph": f"{w.graph_args['kind']} family, {n} DOFs, {Sc} samples, every node"}


def _rel_l2(u, ref, ml):
    u = np.atleast_2d(u)
    ref = np.atleast_2d(ref)
    num = np.sqrt((ml[None, :] * (u - ref) ** 2).sum(axis=1))
    den = np.sqrt((ml[None, :] * ref ** 2).sum(axis=1))
    return float((num / den).max())


def run_grf(args, w, graph):
    import torch
    import paper_2605_02670_gb300 as grf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ne = grf.mesh_elements(graph.lengths, w.h, w.clip)
    G = grf.Graph(graph.edge_u, graph.edge_v, graph.lengths, graph.n_vertices, n_elems=ne)
    S = w.n_samples
    prec = args.precision or w.precision
    out_dtype = "f32" if prec == "mixed" else "f64"
    tsize = 4 if prec == "mixed" else 8
    osz = 4 if out_dtype == "f32" else 8
    out = torch.empty((S, G.n_dofs), dtype=torch.float32 if osz == 4 else torch.float64,
                      device="cuda")
    props = torch.cuda.get_device_properties(local)
    l2_bytes = int(getattr(props, "L2_cache_size", 0) or L2_BYTES)
    n_sm = int(props.multi_processor_count)
    flush = torch.empty(2 * l2_bytes // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    seed0 = rank_seed(w.seed, rank)

    train = None
    if args.precond == "learned":
        # setup outside the timed region: train the network on this workload
        G.precond_init(0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist, npairs = G.precond_train(w.kappa, w.beta, w.k_step, epochs=args.train_epochs,
                                       seed=w.seed)
        torch.cuda.synchronize()
        train = {"epochs": args.train_epochs, "pairs": npairs,
                 "seconds": round(time.perf_counter() - t0, 3),
                 "loss_first": float(hist[0]), "loss_last": float(hist[-1])}
    knobs = {"pcg_layout": args.pcg_layout, "recover_sg": args.recover_sg}
    tune_ms = None
    if args.mass == "consistent":
        # the comparison system runs only on the tensor-core sine-basis
        # interiors; the autotuner times lumped-mass calls, so it is skipped
        if prec != "mixed":
            raise SystemExit("--mass consistent needs mixed precision")
        args.autotune = False
        args.interior = args.interior or "spectral_umma"
    if args.autotune and args.pcg_layout == "auto" and args.recover_sg == 0:
        # launch-schedule autotuner (setup, outside the timed region)
        knobs, tune_ms = G.autotune(w.kappa, w.beta, w.k_step, S, precision=prec,
                                    out_dtype=out_dtype, reps=2, precond=args.precond)
    knobs["precond"] = args.precond
    if args.mass != "lumped":
        knobs["mass"] = args.mass
    if args.interior:
        knobs["interior"] = args.interior
    if args.sweep:
        knobs["sweep"] = args.sweep

    def step(i, timing):
        # phase events (in a replayed graph: event record nodes, recorded by
        # every replay): True = every phase, or a list of phase names
        return G.sample(w.kappa, w.beta, w.k_step, seed0 + i, S, precision=prec,
                        out_dtype=out_dtype, out=out, timing=timing,
                        use_graph=args.use_graph, **knobs)

    # warm-up with every phase timed: the per-phase report and the dominant phase
    warm = []
    for i in range(args.warmup):
        flush.zero_()
        warm.append(step(i, True)[1]["phase_ms"])
    warm = warm[1:] if len(warm) > 1 else warm
    mean_ph = {k: statistics.mean(p[k] for p in warm) for k in warm[0]}
    dom = max(mean_ph, key=mean_ph.get)
    # the timed steps carry the events of the dominant phase only (two event
    # records per call); this untimed call captures that graph
    step(args.warmup, [dom])
    torch.cuda.synchronize()
    times, phases, launches, iters = [], [], [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, st = step(args.warmup + 1 + i, [dom])
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
            phases.append(st["phase_ms"])
            launches.append(st["kernel_launches"])
            iters.append(st)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = statistics.mean(times)
    ms_max = max_over_ranks(ms, dist)
    last_seed = seed0 + args.warmup + args.steps
    accuracy = None
    if not args.no_accuracy:
        accuracy = accuracy_checks(args, w, graph, G, out, last_seed, prec, knobs)
    st = iters[-1]
    L = st["n_nodes"]
    value = job_rate(S, world, ms_max / 1000.0)
    dof_solves = job_rate(G.n_dofs * L * S, world, ms_max / 1000.0)

    # end to end through the C ABI into pinned host memory: the pipelined host
    # entry point (the host copy of one call overlaps the next call's compute),
    # every call's field read back; two host buffers used alternately
    hosts = [torch.empty((S, G.n_dofs), dtype=out.dtype, pin_memory=True) for _ in range(2)]
    hnp = [h.numpy() for h in hosts]
    e2e_opts = grf.make_options(prec, out_dtype, use_graph=args.use_graph, **knobs)
    grf.grf_sample_host_stream(G.handle, w.kappa, w.beta, w.k_step,
                               [seed0 + 9_998, seed0 + 9_999], S, hnp, e2e_opts, stream)  # warm-up
    n_e2e = max(2, min(args.steps, 6))
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grf.grf_sample_host_stream(G.handle, w.kappa, w.beta, w.k_step,
                               [seed0 + 10_000 + i for i in range(n_e2e)], S,
                               [hnp[i % 2] for i in range(n_e2e)], e2e_opts, stream)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / n_e2e, dist)
    # one unpipelined call for comparison (compute, then the whole copy)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grf.grf_sample_host(G.handle, w.kappa, w.beta, w.k_step, seed0 + 20_000, S, hnp[0],
                        e2e_opts, stream)
    e2e_single_s = time.perf_counter() - t0
    del hosts, hnp

    # the roofline phase from the timed steps, the others from the warm-up calls
    mean_ph[dom] = statistics.mean(p[dom] for p in phases)
    how = "event record nodes of the replayed graph" if args.use_graph else "direct calls"
    phase_source = (f"CUDA events on the call's stream ({how}): '{dom}' over the timed "
                    "steps, the other phases over the warm-up calls")
    if rank != 0:
        dist.destroy_process_group()
        return
    hbm_peak, peak_kind = peaks()
    clocks = clk.summary()
    roof = {}
    work, bound = algorithmic(w, G, st, dom, S, tsize, osz, l2_bytes)
    dur_s = mean_ph[dom] / 1000.0
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    fp32_pk = fp32_peak_tflops(sm_mhz, n_sm)
    phases = {}
    for ph, t_ms in mean_ph.items():
        wk, bd = algorithmic(w, G, st, ph, S, tsize, osz, l2_bytes)
        if not wk or not t_ms:
            continue
        if bd == "hbm":
            phases[ph] = {"ms": t_ms, "bound": "hbm", "GB/s": wk / t_ms / 1e6,
                          "frac": wk / t_ms / 1e6 / hbm_peak}
        else:
            phases[ph] = {"ms": t_ms, "bound": "alu", "TFLOP/s": wk / t_ms / 1e9,
                          "frac": wk / t_ms / 1e9 / fp32_pk}
    interior = knobs.get("interior", "spectral" if prec == "mixed" else "thomas")
    spectral = interior in ("spectral", "spectral_tc", "spectral_umma")
    segments = knobs.get("sweep") == "segments"
    kernel_file = {"noise": "noise.cu", "schur": "schur.cu",
                   "condense": ("spectral_mma.cu" if interior == "spectral_tc" else
                                ("dst_gemm.cu" if interior == "spectral_umma" else "spectral.cu"))
                   if spectral else ("thomas.cu" if segments else "sweep.cu"),
                   "pcg": ("pcg_batch.cu" if G.n_kept > 4096 and args.precond == "jacobi" and
                           knobs.get("pcg_layout") != "per_system" else "pcg.cu"),
                   "recover": "spectral.cu" if spectral else
                   ("recover.cu" if segments else "sweep.cu"),
                   "precond_net": "learned.cu"}.get(dom, "api.cu")
    if bound == "hbm":
        ach = work / dur_s / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "peak_source": peak_kind,
                "traffic": traffic_record(kernel_file, w.name)}
    else:
        ach = work / dur_s / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp32_pk,
                "unit": "TFLOP/s", "frac": ach / fp32_pk,
                "peak_source": (f"{n_sm} SMs (device properties) x 128 FP32 lanes x 2 x "
                                f"{sm_mhz:.0f} MHz (median sampled SM clock)"),
                "traffic": traffic_record(kernel_file, w.name)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "kappa": w.kappa, "beta": w.beta, "k_step": w.k_step,
                   "n_dofs": G.n_dofs, "n_vertices": G.n_kept,
                   "n_edges": G.n_edges, "quadrature_nodes": L, "samples_per_gpu": S,
                   "precision": prec,
                   "l2": "flushed between timed device steps; the end-to-end pipeline's "
                         + ("field per call exceeds L2" if S * G.n_dofs * osz > l2_bytes
                            else "field per call fits in L2 (not flushed between its calls)"),
                   "knobs": knobs, "autotune_ms": tune_ms, "cuda_graph": args.use_graph,
                   "training": train,
                   "parallelism": f"replicas x{world}"},
        "dof_solves_per_s": dof_solves,
        "pcg_iters_total": st["pcg_iters_total"], "pcg_iters_max": st["pcg_iters_max"],
        "phase_ms": mean_ph, "phase_ms_source": phase_source,
        "roofline": roof,
        "phase_roofline": phases,
        "accuracy": accuracy,
        "gpu_launches": int(sum(launches)),
        "clocks": clocks,
        "e2e": {"value": job_rate(S, world, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": 3 * 8 * L,
                "d2h_bytes_per_step": S * G.n_dofs * osz,
                "api": f"grf_sample_host_stream, {n_e2e} calls pipelined (host copy of a call "
                       "overlapping the next call's compute), wall time / calls",
                "single_call_value": S / e2e_single_s},
    }
    if accuracy and accuracy.get("fp64_form"):
        line["speedup_vs_fp64_form"] = value / accuracy["fp64_form"]["value"]
    if args.mass != "lumped":
        line["config"]["mass"] = args.mass
    if not args.no_cpu_baseline and world == 1 and args.mass == "lumped":
        # the paper's parallelisation (quadrature nodes over every host core),
        # and beside it the single-thread figure (its instruction counts are
        # single-threaded)
        cb1 = oracle_sample(w, graph)
        cb1.pop("wall_s", None)
        cbp = oracle_sample(w, graph, parallel=True)
        cbp.pop("wall_s", None)
        line["cpu_baseline"] = cbp
        line["cpu_baseline_1core"] = cb1
        if accuracy and "_check" in accuracy:
            accuracy["reduced_vs_oracle"] = oracle_check(w, accuracy["_check"])
            line["rel_l2"] = {"vs_oracle_small_graph": accuracy["reduced_vs_oracle"]["rel_l2"]}
            if "full_vs_fp64_form" in accuracy:
                line["rel_l2"]["vs_fp64_form_full_size"] = \
                    accuracy["full_vs_fp64_form"]["rel_l2"]
    if accuracy:
        accuracy.pop("_check", None)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="grf", choices=["grf", "reference"])
    ap.add_argument("--workload", default="grid300", choices=sorted(gi.WORKLOADS))
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy checks (oracle on a small graph, FP64 form)")
    ap.add_argument("--pcg-layout", default="auto", choices=["auto", "per_system", "staged", "staged_pairs",
                                                          "batched"])
    ap.add_argument("--recover-sg", type=int, default=0, choices=[0, 1, 2, 4])
    ap.add_argument("--interior", default=None, choices=[None, "thomas", "spectral", "spectral_tc", "spectral_umma"],
                    help="edge-interior solver (default: the autotuner's or the library's)")
    ap.add_argument("--sweep", default=None, choices=[None, "segments", "nodes"],
                    help="layout of the FP32 tridiagonal sweeps (default: the library's)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--no-graph", dest="use_graph", action="store_false",
                    help="direct calls instead of replaying each call as a captured CUDA graph")
    ap.add_argument("--mass", default="lumped", choices=["lumped", "consistent"],
                    help="mass matrix of noise and operator: the method's lumped mass, or "
                         "the consistent-mass comparison system (mixed precision)")
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "neumann", "learned"],
                    help="vertex PCG preconditioner (mixed precision for learned; the "
                         "learned network is trained on the workload before timing)")
    ap.add_argument("--train-epochs", type=int, default=40)
    ap.add_argument("--kappa", type=float, default=None,
                    help="override the workload's kappa (same graph and mesh)")
    ap.add_argument("--beta", type=float, default=None,
                    help="override the workload's beta (same graph and mesh)")
    args = ap.parse_args()
    w = gi.WORKLOADS[args.workload]
    if args.kappa is not None or args.beta is not None:
        w = dataclasses.replace(w, kappa=w.kappa if args.kappa is None else args.kappa,
                                beta=w.beta if args.beta is None else args.beta)
    graph = w.graph()
    if args.impl == "reference":
        run_reference(args, w, graph)
    else:
        run_grf(args, w, graph)


if __name__ == "__main__":
    main()
