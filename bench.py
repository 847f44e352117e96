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


def oracle_sample(w, graph, n_nodes_sample=4):
    """Time the FP64 oracle on a bounded sample of the workload: mesh and
    assembly, noise for all samples, and `n_nodes_sample` of the L quadrature
    nodes (spread over the range), each factorised once and solved for every
    sample. Extrapolated linearly in the node count."""
    from oracle import fem, noise, quadrature, sampler
    t0 = time.perf_counter()
    ne = None
    if w.clip:
        ne = np.clip(np.ceil(graph.lengths / w.h), *w.clip)
    mesh = fem.build_mesh(graph.edge_u, graph.edge_v, graph.lengths, graph.n_vertices, h=w.h,
                          n_elems=ne)
    ml, _, kmat = sampler.assemble(mesh, w.kappa)
    b = noise.white_noise(ml, w.seed, w.n_samples)
    t_fixed = time.perf_counter() - t0
    f = w.beta - math.floor(w.beta)
    t, wt = quadrature.nodes(f, w.k_step)
    pick = np.linspace(0, len(t) - 1, n_nodes_sample).round().astype(int)
    t1 = time.perf_counter()
    for i in pick:
        sampler.shifted_sum(ml, kmat, b, [t[i]], [wt[i]])
    t_nodes = time.perf_counter() - t1
    total = t_fixed + t_nodes * len(t) / len(pick)
    return {"value": w.n_samples / total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{w.name}: mesh+assembly+noise for {w.n_samples} samples, then "
                       f"{len(pick)} of {len(t)} quadrature nodes (SuperLU factorisation + "
                       f"{w.n_samples} solves each, single thread), extrapolated linearly "
                       f"to all nodes; measured {t_fixed + t_nodes:.1f} s")}


def run_reference(args, w, graph):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # the oracle keeps no state between calls, so it needs no warm-up;
    # every step is one timed bounded sample
    vals = []
    cb = None
    for _ in range(args.steps):
        cb = oracle_sample(w, graph, n_nodes_sample=2)
        vals.append(cb["value"])
    v = statistics.median(vals)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * w.n_samples / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name}, "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU path


def algorithmic(w, G, stats, phase, S, tsize, out_size):
    """Algorithmic bytes (or flops) of one launch of a phase, from the
    per-unit figures: noise writes N S values and reads N mass factors; one
    PCG iteration of one system moves ~10 |V| FP64 vector values and each
    (node, sample-batch) reads the Schur matrix ((|V| + 2|E|) values + 2|E|
    indices); recovery reads the noise, the vertex solutions and writes U."""
    N, V, E, NI = G.n_dofs, G.n_kept, G.n_edges, G.n_interior
    L = stats["n_nodes"]
    if phase == "noise":
        return N * S * tsize + N * 8, "hbm"
    if phase == "pcg":
        it = stats["pcg_iters_total"]
        if L * S * V * 8 <= L2_BYTES:
            # the vertex vectors of every system stay on chip (shared memory and
            # registers of the sample-group layout): bounded by the FP32 work,
            # SpMV 2 (|V| + 2|E|) + dots and updates ~10 |V| flops per iteration
            return it * (2 * (V + 2 * E) + 10 * V), "alu"
        return it * 10 * V * 8 + (it / S) * ((V + 2 * E) * 8 + 2 * E * 4), "hbm"
    if phase == "recover":
        # FP32 FMA work: ~6 flops per (interior node, quadrature node, sample)
        return 6.0 * NI * L * S, "alu"
    if phase == "condense":
        return 4.0 * NI * L * S, "alu"
    if phase == "schur":
        return L * (E * 16 + V * 8 + 2 * E * 8), "hbm"
    return 0, "hbm"


def fp32_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flops (FMA) per clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


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
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
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
    if args.autotune and args.pcg_layout == "auto" and args.recover_sg == 0:
        # launch-schedule autotuner (setup, outside the timed region)
        knobs, tune_ms = G.autotune(w.kappa, w.beta, w.k_step, S, precision=prec,
                                    out_dtype=out_dtype, reps=2, precond=args.precond)
    knobs["precond"] = args.precond
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
    st = iters[-1]
    L = st["n_nodes"]
    value = job_rate(S, world, ms_max / 1000.0)
    dof_solves = job_rate(G.n_dofs * L * S, world, ms_max / 1000.0)

    # end to end through the C ABI with a host output buffer
    host = torch.empty((S, G.n_dofs), dtype=out.dtype, pin_memory=True)
    e2e_opts = grf.make_options(prec, out_dtype, use_graph=args.use_graph, **knobs)
    grf.grf_sample_host(G.handle, w.kappa, w.beta, w.k_step, seed0 + 9_999, S, host.numpy(),
                        e2e_opts, stream)  # warm-up (captures the graph for this buffer)
    e2e_t = []
    for i in range(max(1, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grf.grf_sample_host(G.handle, w.kappa, w.beta, w.k_step, seed0 + 10_000 + i, S,
                            host.numpy(), e2e_opts, stream)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.mean(e2e_t), dist)

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
    work, bound = algorithmic(w, G, st, dom, S, tsize, osz)
    dur_s = mean_ph[dom] / 1000.0
    interior = knobs.get("interior", "spectral" if prec == "mixed" else "thomas")
    spectral = interior in ("spectral", "spectral_tc")
    segments = knobs.get("sweep") == "segments"
    kernel_file = {"noise": "noise.cu", "schur": "schur.cu",
                   "condense": ("spectral_mma.cu" if interior == "spectral_tc" else "spectral.cu")
                   if spectral else ("thomas.cu" if segments else "sweep.cu"),
                   "pcg": "pcg.cu", "recover": "spectral.cu" if spectral else
                   ("recover.cu" if segments else "sweep.cu"),
                   "precond_net": "learned.cu"}.get(dom, "api.cu")
    if bound == "hbm":
        ach = work / dur_s / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "peak_source": peak_kind,
                "traffic": traffic_record(kernel_file, w.name)}
    else:
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        pk = fp32_peak_tflops(mhz)
        ach = work / dur_s / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz",
                "traffic": traffic_record(kernel_file, w.name)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "n_dofs": G.n_dofs, "n_vertices": G.n_kept,
                   "n_edges": G.n_edges, "quadrature_nodes": L, "samples_per_gpu": S,
                   "precision": prec, "l2": "flushed between timed steps",
                   "knobs": knobs, "autotune_ms": tune_ms, "cuda_graph": args.use_graph,
                   "training": train,
                   "parallelism": f"replicas x{world}"},
        "dof_solves_per_s": dof_solves,
        "pcg_iters_total": st["pcg_iters_total"], "pcg_iters_max": st["pcg_iters_max"],
        "phase_ms": mean_ph, "phase_ms_source": phase_source,
        "roofline": roof,
        "gpu_launches": int(sum(launches)),
        "clocks": clocks,
        "e2e": {"value": job_rate(S, world, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": 3 * 8 * L,
                "d2h_bytes_per_step": S * G.n_dofs * osz},
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = oracle_sample(w, graph)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="grf", choices=["grf", "reference"])
    ap.add_argument("--workload", default="rgg2000", choices=sorted(gi.WORKLOADS))
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pcg-layout", default="auto", choices=["auto", "per_system", "staged", "staged_pairs"])
    ap.add_argument("--recover-sg", type=int, default=0, choices=[0, 1, 2, 4])
    ap.add_argument("--interior", default=None, choices=[None, "thomas", "spectral", "spectral_tc"],
                    help="edge-interior solver (default: the autotuner's or the library's)")
    ap.add_argument("--sweep", default=None, choices=[None, "segments", "nodes"],
                    help="layout of the FP32 tridiagonal sweeps (default: the library's)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--no-graph", dest="use_graph", action="store_false",
                    help="direct calls instead of replaying each call as a captured CUDA graph")
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "neumann", "learned"],
                    help="vertex PCG preconditioner (mixed precision for learned; the "
                         "learned network is trained on the workload before timing)")
    ap.add_argument("--train-epochs", type=int, default=40)
    args = ap.parse_args()
    w = gi.WORKLOADS[args.workload]
    graph = w.graph()
    if args.impl == "reference":
        run_reference(args, w, graph)
    else:
        run_grf(args, w, graph)


if __name__ == "__main__":
    main()
