"""The multi-rank path of bench.py on CPU: world size 2 over gloo.

With N > 1 GPUs every rank runs an independent replica of the sampler on its own
seed (no collective on the data path); the job's time is the slowest rank's and
its throughput counts every rank's samples. These are the host-side pieces of
that path: the all-reduce of the timings, the per-rank seeds (distinct noise
streams, checked with the oracle's Philox generator) and the job-rate formula."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank: int, world: int, port: int, out_q) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from oracle import noise

        ms_local = 10.0 + 5.0 * rank
        ms_max = bench.max_over_ranks(ms_local, dist, device="cpu")
        seed = bench.rank_seed(1, rank)
        b = noise.white_noise(np.ones(8), seed, 2)
        out_q.put((rank, ms_max, seed, b.tolist()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_the_slowest_time_and_draw_distinct_samples():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 15.0 for r in res)  # every rank sees the slowest rank's time
    assert res[0][2] != res[1][2]
    assert not np.allclose(res[0][3], res[1][3])  # independent replicas


def test_job_rate_counts_every_rank():
    import bench

    assert bench.job_rate(16, 2, 0.015) == pytest.approx(16 * 2 / 0.015)
    assert bench.job_rate(16, 1, 0.003) == pytest.approx(16 / 0.003)
    assert bench.max_over_ranks(3.5) == 3.5  # one rank: no process group
