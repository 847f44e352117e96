"""Host-side arithmetic of bench.py's roofline object, on CPU: the FP32 peak
from the unit counts and clock, the algorithmic work of each phase from its
per-unit figure, and the traffic record that is valid only for the kernel
source it was measured on. The expected values are worked out here by hand
from the per-unit figures (not by calling the same expressions). Also the
reference arm's contract line (it runs the oracle on the host cores only)."""
import hashlib
import json
import os
from types import SimpleNamespace

import pytest

import bench


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA at 2070 MHz = 80.54784 TFLOP/s
    assert bench.fp32_peak_tflops(2070) == pytest.approx(80.54784, rel=1e-12)
    assert bench.fp32_peak_tflops(1000) == pytest.approx(38.912, rel=1e-12)
    # the SM count is an argument (read from the device by the bench)
    assert bench.fp32_peak_tflops(1000, n_sm=100) == pytest.approx(25.6, rel=1e-12)


def _workload(V=1980, E=4990, NI=957_699):
    return SimpleNamespace(n_dofs=V + NI, n_kept=V, n_edges=E, n_interior=NI)


def test_pcg_work_on_chip_counts_flops():
    G = _workload()
    stats = {"n_nodes": 148, "pcg_iters_total": 90_592}
    work, bound = bench.algorithmic(None, G, stats, "pcg", 16, 4, 4)
    # per iteration: SpMV 4 (1980 + 2 * 4990) = 47 840 flops, vector work 10 * 1980
    assert bound == "alu"
    assert work == 90_592 * (47_840 + 19_800)


def test_pcg_work_off_chip_counts_bytes():
    G = _workload(V=20_000, E=59_991, NI=48_000_000)
    stats = {"n_nodes": 148, "pcg_iters_total": 145_235}
    S = 64  # 148 x 64 x 20 000 x 8 B = 1.5 GB of vertex vectors: larger than L2
    for tsize in (4, 8):
        work, bound = bench.algorithmic(None, G, stats, "pcg", S, tsize, 4)
        vectors = 145_235 * 10 * 20_000 * tsize
        matrix = (145_235 / 64) * (20_000 + 59_991) * 12
        assert bound == "hbm"
        assert work == pytest.approx(vectors + matrix, rel=1e-12)
    # the same graph with a 2 GB L2 keeps the vectors on chip
    work, bound = bench.algorithmic(None, G, stats, "pcg", S, 4, 4, l2_bytes=2 << 30)
    assert bound == "alu"


def test_noise_recovery_condensation_and_schur_work():
    G = _workload(V=10, E=12, NI=1000)
    stats = {"n_nodes": 7, "pcg_iters_total": 0}
    S = 3
    assert bench.algorithmic(None, G, stats, "noise", S, 4, 4) == (1010 * 3 * 4 + 1010 * 4, "hbm")
    # condensation + recovery: 12 flops per (interior node, node, sample), 4 + 8
    assert bench.algorithmic(None, G, stats, "recover", S, 4, 4) == (8.0 * 1000 * 7 * 3, "alu")
    assert bench.algorithmic(None, G, stats, "condense", S, 4, 4) == (4.0 * 1000 * 7 * 3, "alu")
    # per node: 2 FP64 words per edge block pair, the vertex diagonal, 2 off-diagonals per edge
    assert bench.algorithmic(None, G, stats, "schur", S, 4, 4) == (7 * (12 * 16 + 10 * 8 + 24 * 8),
                                                                    "hbm")


def test_lumped_mass_weights_in_dof_order():
    import numpy as np
    # a path 0 - 1 - 2 plus an isolated input vertex 3 (dropped by the library)
    graph = SimpleNamespace(edge_u=np.array([0, 1]), edge_v=np.array([1, 2]),
                            lengths=np.array([1.0, 0.5]))
    G = SimpleNamespace(vertex_map=np.array([0, 1, 2, -1]), n_kept=3)
    ne = np.array([4, 2])
    ml = bench.ml_weights(graph, ne, G)
    # vertices: 0.25/2, 0.25/2 + 0.25/2, 0.25/2; interiors: 3 x 0.25, 1 x 0.25
    np.testing.assert_allclose(ml, [0.125, 0.25, 0.125, 0.25, 0.25, 0.25, 0.25])
    assert ml.sum() == pytest.approx(1.5)


def test_oracle_stands_in_a_smaller_graph_of_the_family():
    w = bench.gi.WORKLOADS["grid300"]
    g, mesh, scale = bench.oracle_graph(w, w.graph())
    assert mesh.n_dofs <= bench.ORACLE_MAX_DOFS and scale > 30
    w2 = bench.gi.WORKLOADS["square5"]
    g2, mesh2, scale2 = bench.oracle_graph(w2, w2.graph())
    assert scale2 == 1.0 and mesh2.n_dofs == 550


def test_traffic_record_only_for_the_measured_source():
    p = os.path.join(bench.ROOT, "profiles", "traffic.json")
    recs = json.load(open(p))
    assert bench.traffic_record("pcg.cu", "no_such_workload") is None
    for key, rec in recs.items():
        kernel_file, workload = key.split(":")
        src = os.path.join(bench.ROOT, "paper_2605_02670_gb300", "csrc", kernel_file)
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        expect = rec["bytes_per_launch"] if sha == rec["sha256"] else None
        assert bench.traffic_record(kernel_file, workload) == expect
        assert rec["bytes_per_launch"] > 0


def _run_bench(args, env_extra=None):
    import subprocess
    import sys

    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py")] + args,
                          capture_output=True, text=True, env=env, timeout=300)


def test_reference_arm_prints_one_contract_line():
    """The reference arm (the FP64 oracle on the host cores, bounded samples):
    one JSON line with the keys of the bench contract, its e2e equal to its
    value with no host-device copies."""
    r = _run_bench(["--impl", "reference", "--workload", "square5", "--steps", "2",
                    "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    # ms_per_step is what one step took (one bounded oracle sample)
    assert 0 < d["ms_per_step"] < 300_000 and d["ms_per_step_is"]
    assert d["config"]["workload"] == "square5"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    r = _run_bench(["--impl", "reference", "--workload", "square5", "--steps", "1",
                    "--warmup", "1"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
