"""The z-slab decomposition and the gradient sum on gloo ranks (CPU).

Every rank sweeps its slab with the FP64 oracle and exchanges r halo planes
with its neighbours; the slabs put together must equal the oracle's sweeps
of the whole grid exactly (each point sees the same FP64 inputs in the same
order).  Shots split across ranks and summed must give the gradient of all
shots in one process.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_2507_11067_gb300 import distributed as mdist  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case_grid(case):
    shape, r, n, steps, overlap = case
    grid = workloads.uniform_grid(*n, r, workload=2, salt=900 + r).astype(np.float64)
    # a nonzero outer halo: the global boundary values must stay as they are
    grid[:r] = 0.5
    grid[-r:] = -0.25
    c = workloads.normal_coeffs(shape, r, workload=2, salt=900 + r)
    return grid, c


def _oracle_sweep(shape, r, c):
    def sweep(padded_in, out):
        out.copy_(torch.from_numpy(oracle.stencil(shape, r, c, padded_in.numpy())))
    return sweep


def _sweep_worker(rank, world, port, cases, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for k, case in enumerate(cases):
            shape, r, n, steps, overlap = case
            grid, c = _case_grid(case)
            ss = mdist.SlabSweep(shape, r, c, *n, sweep=_oracle_sweep(shape, r, c))
            slab = ss.local_slab(torch.from_numpy(grid)).clone()
            # the halo planes inside the grid start as garbage: the first
            # exchange must overwrite them
            if rank > 0:
                slab[:r] = 1e30
            if rank < world - 1:
                slab[-r:] = 1e30
            res = ss.iterate(slab, steps, overlap=overlap)
            q.put((k, rank, ss.z0, ss.z1, res.numpy().copy()))
    except Exception as e:          # reported to the parent instead of leaving it waiting
        q.put(("error", rank, repr(e), None, None))
    finally:
        dist.destroy_process_group()


def _run(world, target, args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port) + args + (q,)) for r in range(world)]
    for p in procs:
        p.start()
    return ctx, q, procs


CASES = [
    ("star", 2, (13, 10, 11), 3, True),
    ("star", 2, (13, 10, 11), 3, False),
    ("box", 1, (9, 8, 14), 4, True),
    ("star", 4, (12, 9, 20), 2, True),
    ("star", 2, (8, 7, 8), 2, True),     # 3 or 4 ranks get slabs of 2-3 planes: thinner than 2r, no split
]


@pytest.mark.parametrize("world", [2, 3, 4])
def test_slabs_equal_the_single_domain_sweeps(world):
    cases = CASES
    ctx, q, procs = _run(world, _sweep_worker, (cases,))
    got = []
    try:
        while len(got) < world * len(cases):
            item = q.get(timeout=300)
            assert item[0] != "error", item
            got.append(item)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for k, case in enumerate(cases):
        shape, r, n, steps, overlap = case
        grid, c = _case_grid(case)
        ref = grid.copy()
        for _ in range(steps):
            ref[r:-r, r:-r, r:-r] = oracle.stencil(shape, r, c, ref)
        parts = sorted((g for g in got if g[0] == k), key=lambda g: g[1])
        assert [p[1] for p in parts] == list(range(world))
        z = 0
        for _, rank, z0, z1, slab in parts:
            assert z0 == z and z1 > z0
            z = z1
            # the slab's interior planes and both halos equal the global
            # result there (the halos after the last exchange)
            np.testing.assert_array_equal(slab, ref[z0:z1 + 2 * r], err_msg=f"{case} rank {rank}")
        assert z == n[2]


def test_slab_bounds_cover_the_grid():
    for nz in (1, 7, 8, 513, 1024):
        for world in (1, 2, 3, 4, 8):
            b = [mdist.slab_bounds(nz, world, k) for k in range(world)]
            assert b[0][0] == 0 and b[-1][1] == nz
            assert all(b[k][1] == b[k + 1][0] for k in range(world - 1))
            sizes = [z1 - z0 for z0, z1 in b]
            assert max(sizes) - min(sizes) <= 1


def test_thin_slabs_and_planar_shapes_are_refused():
    class One:
        @staticmethod
        def get_world_size(group=None):
            return 4

        @staticmethod
        def get_rank(group=None):
            return 0

    with pytest.raises(ValueError, match="thinner"):
        mdist.SlabSweep("star", 4, np.zeros(27), 8, 8, 12, comm=One, sweep=lambda a, b: None)
    with pytest.raises(ValueError, match="star or box"):
        mdist.SlabSweep("star2d", 1, np.zeros(6), 8, 8, 12, comm=One, sweep=lambda a, b: None)


# ---------------------------------------------------------------- gradients

R = 4
NSTEPS = 24
SHOTS = [(3, 4, 5), (8, 6, 4), (5, 9, 7), (6, 3, 8)]


def _wave(shots):
    nz, ny, nx = 11, 12, 10
    g = np.random.default_rng(5)
    v = 2000.0 * (1.0 + 0.1 * g.uniform(-1, 1, size=(nz, ny, nx)))
    h, dt = 10.0, 0.4 * 10.0 / float(np.max(v))
    t = np.arange(NSTEPS) * dt
    amp = np.zeros((NSTEPS, len(shots)))
    amp[:, :] = (dt * dt * workloads.ricker(t, 60.0, 1.0 / 60.0))[:, None]
    return oracle.WaveProblem(R, oracle.fd2_star_coeffs(R), oracle.model_m(v, dt, h), (3, 0.1),
                              shots, amp, zrec=2)


def _gradient(shots):
    p = _wave(shots)
    rec, states = p.forward(NSTEPS, keep_states=True)
    return p.gradient_m(rec, states)          # J = 1/2 |d|^2: the residual is the record


def _grad_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = SHOTS[rank::world]
        g = torch.from_numpy(_gradient(mine))
        mdist.allreduce_gradient(g)
        q.put((rank, g.numpy().copy()))
        with pytest.raises(ValueError):
            mdist.allreduce_gradient(g.float())
    finally:
        dist.destroy_process_group()


def test_shot_gradients_summed_across_ranks_equal_all_shots():
    world = 2
    ctx, q, procs = _run(world, _grad_worker, ())
    try:
        got = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    full = _gradient(SHOTS)
    assert np.abs(full).max() > 0
    for rank, g in got:
        np.testing.assert_allclose(g, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    np.testing.assert_array_equal(got[0][1], got[1][1])
