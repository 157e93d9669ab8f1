"""Sweeps and gradients across ranks (one process per GPU, torch.distributed).

A grid split into z-slabs: every rank keeps its slab of the padded grid --
its own planes plus r halo planes on each side -- and, before each sweep,
refreshes the halo planes that lie inside the global grid from its
neighbours with one point-to-point exchange (r planes each way; NCCL on
GPUs).  The outer halo of the first and last rank is the global grid's own
halo and is never exchanged.  This is the paper's multi-process layer
(Sec. 4.6: domain decomposition with halo exchange between processes) in
the GB300 setting: the exchange is device-to-device, the sweep is the
library's.

Acoustic shots are independent: ranks own disjoint shots of one velocity
model, and the only collective is the final FP64 sum of their gradients
(``allreduce_gradient``).
"""
from __future__ import annotations

import torch


def slab_bounds(nz: int, world: int, rank: int):
    """[z0, z1) of rank's planes: nz split as evenly as possible, the first
    nz % world ranks one plane more."""
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


class SlabSweep:
    """Iterated sweeps of one stencil on a z-slab decomposition.

    shape, r: the 3D stencil (star or box); nx, ny, nz: the global interior;
    group: the process group (None = the default group); sweep: the function
    computing a slab's interior from its padded planes,
    ``sweep(padded_in, out)`` with ``padded_in`` (nzl+2r, ny+2r, nx+2r) and
    ``out`` (nzl, ny, nx) -- the library's own sweep by default; comm: the
    point-to-point layer, ``torch.distributed`` by default (any object with
    its get_world_size / get_rank / get_global_rank / P2POp / isend / irecv /
    batch_isend_irecv interface).
    """

    def __init__(self, shape: str, r: int, coeffs, nx: int, ny: int, nz: int, group=None, sweep=None,
                 path: str = "auto", comm=None):
        if shape not in ("star", "box"):
            raise ValueError("slab sweeps split 3D grids along z: shape must be star or box")
        if comm is None:
            import torch.distributed as comm
        dist = self.dist = comm
        self.shape, self.r, self.coeffs = shape, int(r), coeffs
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.z0, self.z1 = slab_bounds(self.nz, self.world, self.rank)
        if self.z1 - self.z0 < self.r and self.world > 1:
            raise ValueError(f"slab of {self.z1 - self.z0} planes is thinner than the radius {self.r}")
        if sweep is None:
            from . import _lib

            def sweep(padded_in, out):
                _lib.apply(shape, self.r, coeffs, padded_in, out, path=path)
        self.sweep = sweep

    @property
    def nzl(self) -> int:
        return self.z1 - self.z0

    def local_slab(self, global_padded):
        """This rank's padded slab (nzl+2r planes) cut from a global padded
        grid (nz+2r, ny+2r, nx+2r)."""
        return global_padded[self.z0:self.z1 + 2 * self.r]

    def _peer(self, rank):
        return rank if self.group is None else self.dist.get_global_rank(self.group, rank)

    def _post(self, slab):
        """Start the exchange of `slab`'s edge planes: send its first and
        last r interior planes, receive the neighbours' into buffers.
        Returns (requests, [(halo slice, buffer)])."""
        r, nzl = self.r, self.nzl
        ops, recv = [], []
        if self.rank > 0:          # lower neighbour: my first r planes go down, its last r come up
            lo = self._peer(self.rank - 1)
            ops.append(self.dist.P2POp(self.dist.isend, slab[r:2 * r].contiguous(), lo, self.group))
            buf = torch.empty_like(slab[0:r])
            ops.append(self.dist.P2POp(self.dist.irecv, buf, lo, self.group))
            recv.append((slice(0, r), buf))
        if self.rank < self.world - 1:
            hi = self._peer(self.rank + 1)
            ops.append(self.dist.P2POp(self.dist.isend, slab[nzl:nzl + r].contiguous(), hi, self.group))
            buf = torch.empty_like(slab[nzl + r:nzl + 2 * r])
            ops.append(self.dist.P2POp(self.dist.irecv, buf, hi, self.group))
            recv.append((slice(nzl + r, nzl + 2 * r), buf))
        reqs = self.dist.batch_isend_irecv(ops) if ops else []
        return reqs, recv

    @staticmethod
    def _finish(slab, pending):
        reqs, recv = pending
        for req in reqs:
            req.wait()
        for sl, buf in recv:
            slab[sl].copy_(buf)

    def exchange(self, slab):
        """Refresh the halo planes of `slab` (in place) from the neighbours'
        edge planes: r planes to and from each neighbour."""
        self._finish(slab, self._post(slab))

    def _sweep_planes(self, src, dst, z0, z1):
        """dst's interior planes [z0, z1) from src (both padded slabs)."""
        r = self.r
        if z1 > z0:
            self.sweep(src[z0:z1 + 2 * r], dst[r + z0:r + z1, r:r + self.ny, r:r + self.nx])

    def iterate(self, slab, steps: int, overlap: bool = True):
        """`steps` sweeps u <- S(u) of the rank's padded slab; returns the
        slab holding the result (a second buffer alternates with `slab`).

        With `overlap`, each sweep first computes the r edge planes at each
        end, starts their exchange, computes the inner planes while the
        halos travel, then waits: the exchange of one layer hidden behind the
        compute of the others, as in the paper's z-layer pipeline (Sec. 4.6,
        Fig. 9).  Without it (or when the slab is thinner than 2r planes),
        the whole slab is computed and then exchanged.  The global outer
        halo and the x, y halos are kept as they are."""
        r, nzl = self.r, self.nzl
        cur, nxt = slab, slab.clone()
        self.exchange(cur)
        split = overlap and self.world > 1 and nzl >= 2 * r
        for _ in range(steps):
            if split:
                self._sweep_planes(cur, nxt, 0, r)
                self._sweep_planes(cur, nxt, nzl - r, nzl)
                pending = self._post(nxt)
                self._sweep_planes(cur, nxt, r, nzl - r)
                self._finish(nxt, pending)
            else:
                self._sweep_planes(cur, nxt, 0, nzl)
                self.exchange(nxt)
            cur, nxt = nxt, cur
        return cur


def allreduce_gradient(grad, group=None):
    """Sum the ranks' gradients (FP64) in place: each rank ran its own shots
    of the same model."""
    import torch.distributed as dist
    if grad.dtype != torch.float64:
        raise ValueError("gradients are accumulated in FP64")
    dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad
