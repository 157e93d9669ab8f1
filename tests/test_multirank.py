"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
seeded inputs (weak scaling, no collective on the data path), timed as the
slowest rank, reported as the whole job's rate."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import workloads  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        box = bench.sweep_input("box", 1, 8, rank)
        star = bench.sweep_input("star", 4, 8, rank)
        wave = workloads.WaveInputs(48, 48, 48, nshots=2, nsteps=4, workload=4, sponge=6, salt=rank)
        mine = torch.tensor([float(np.float64(box).sum()), float(np.float64(star).sum())], dtype=torch.float64)
        every = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(every, mine)
        # rank 1 is the slow one
        slowest = bench.max_over_ranks(1.0 + 0.5 * rank, dist, torch.device("cpu"))
        q.put((rank, [t.tolist() for t in every], slowest, [list(p) for p in wave.src]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_inputs_and_time_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    (r0, seen0, slow0, src0), (r1, seen1, slow1, src1) = res
    # both ranks agree on every rank's inputs and on the job time (the slowest rank's)
    assert seen0 == seen1 and slow0 == slow1 == 1.5
    # the ranks' inputs are different seeded problems ...
    assert seen0[0] != seen0[1]
    assert src0 != src1
    # ... and each is the one a single process makes for that rank
    for rank in (0, 1):
        assert seen0[rank][0] == float(np.float64(bench.sweep_input("box", 1, 8, rank)).sum())
        assert seen0[rank][1] == float(np.float64(bench.sweep_input("star", 4, 8, rank)).sum())


def test_job_rate_counts_every_rank_over_the_slowest_time():
    assert bench.job_rate(2, 3e9, 1.5) == pytest.approx(4.0)
    assert bench.job_rate(1, 1e9, 0.5) == pytest.approx(2.0)
    assert bench.max_over_ranks(0.25, None, None) == 0.25
