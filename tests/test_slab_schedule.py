"""The order of work in one rank's slab sweep (the z-layer pipeline of the
paper's Sec. 4.6, Fig. 9), on a recording communicator: with overlap, the r
edge planes at each end are computed first, their exchange is started, the
inner planes are computed while it is in flight, and only then is it waited
for; the planes sent are the ones this step just computed, and the planes
received land in the halo.  Without overlap the whole slab is computed
before the exchange starts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_11067_gb300 import distributed as mdist  # noqa: E402


class Comm:
    """A stand-in for torch.distributed with a log of what was called."""

    def __init__(self, world, rank, log):
        self.world, self.rank, self.log = world, rank, log

    def get_world_size(self, group=None):
        return self.world

    def get_rank(self, group=None):
        return self.rank

    def get_global_rank(self, group, rank):
        return rank

    def isend(self):          # only identities: P2POp names which one
        pass

    def irecv(self):
        pass

    class P2POp:
        def __init__(self, op, tensor, peer, group=None):
            self.op, self.tensor, self.peer = op, tensor, peer

    def batch_isend_irecv(self, ops):
        log = self.log

        class Req:
            def __init__(self, op):
                self.op = op

            def wait(self):
                log.append(("wait", self.op.peer))
                if self.op.op.__name__ == "irecv":
                    self.op.tensor.fill_(1000.0 + self.op.peer)   # the peer's planes arrive

        for op in ops:
            kind = "send" if op.op.__name__ == "isend" else "recv"
            log.append((kind, op.peer, op.tensor.clone()))
        return [Req(op) for op in ops]


def _run(world, rank, nz, r, steps, overlap):
    log = []
    comm = Comm(world, rank, log)
    counter = {"step": 0}

    def sweep(padded_in, out):
        # mark each computed plane with (step, plane within this call)
        k = counter["step"]
        z0 = out.storage_offset() // out.stride(0) - r   # interior plane index of out[0]
        for i in range(out.shape[0]):
            out[i] = 10.0 * k + (z0 + i) / 100.0
        log.append(("sweep", z0, z0 + out.shape[0]))

    nx = ny = 4
    ss = mdist.SlabSweep("star", r, np.zeros(3 * (2 * r + 1)), nx, ny, nz, comm=comm, sweep=sweep)
    slab = torch.zeros((ss.nzl + 2 * r, ny + 2 * r, nx + 2 * r), dtype=torch.float64)
    out = None
    for k in range(steps):
        counter["step"] = k
        out = ss.iterate(slab if out is None else out, 1, overlap=overlap)
    return ss, log, out


def _events(log):
    return [e[0] if e[0] != "sweep" else ("sweep", e[1], e[2]) for e in log]


@pytest.mark.parametrize("overlap", [True, False])
def test_middle_rank_schedule(overlap):
    r, nz, world, rank = 2, 30, 3, 1          # slab of 10 planes, both neighbours
    ss, log, out = _run(world, rank, nz, r, 1, overlap)
    nzl = ss.nzl
    ev = _events(log)
    # the initial halo exchange of the input comes first
    first_sweep = next(i for i, e in enumerate(ev) if isinstance(e, tuple))
    assert ev[:first_sweep].count("send") == 2 and ev[:first_sweep].count("wait") == 4
    rest = ev[first_sweep:]
    if overlap:
        assert rest[0] == ("sweep", 0, r) and rest[1] == ("sweep", nzl - r, nzl)
        assert rest[2:6].count("send") == 2 and rest[2:6].count("recv") == 2
        assert rest[6] == ("sweep", r, nzl - r)            # inner planes while the halos travel
        assert rest[7:] == ["wait"] * 4
    else:
        assert rest[0] == ("sweep", 0, nzl)
        assert rest[1:5].count("send") == 2 and rest[5:] == ["wait"] * 4
    # what was sent after the sweep: this step's edge planes (marker 10*0 + z/100)
    sends = [e for e in log if e[0] == "send"][2:]
    by_peer = {e[1]: e[2] for e in sends}
    lo = by_peer[rank - 1][:, r, r].numpy()
    hi = by_peer[rank + 1][:, r, r].numpy()
    np.testing.assert_allclose(lo, [z / 100.0 for z in range(0, r)])
    np.testing.assert_allclose(hi, [z / 100.0 for z in range(nzl - r, nzl)])
    # and the received planes are in the halo
    assert torch.all(out[:r] == 1000.0 + rank - 1) and torch.all(out[nzl + r:] == 1000.0 + rank + 1)


def test_end_ranks_talk_to_one_neighbour():
    r, nz, world = 1, 12, 3
    for rank, peers in ((0, {1}), (2, {1})):
        _, log, out = _run(world, rank, nz, r, 2, True)
        assert {e[1] for e in log if e[0] in ("send", "recv")} == peers
        # the outer halo of the global grid is never overwritten
        if rank == 0:
            assert torch.all(out[:r] == 0.0)
        else:
            assert torch.all(out[-r:] == 0.0)


def test_thin_slab_does_not_split():
    r, nz, world, rank = 2, 9, 3, 1           # 3 planes < 2r: whole slab, then exchange
    ss, log, _ = _run(world, rank, nz, r, 1, True)
    sweeps = [e for e in log if e[0] == "sweep"]
    assert sweeps == [("sweep", 0, ss.nzl)]
