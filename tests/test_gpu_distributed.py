"""The z-slab decomposition with the library's own sweeps on one GPU.

Ranks are threads of one process joined by an in-process mailbox in place of
torch.distributed: the waits are on the host, every kernel is the library's
stencil sweep on strided sub-slab views (edge planes, then inner planes while
the halos travel).  The slabs put together must match the library's sweeps
of the whole grid and the FP64 oracle.
"""
import queue
import threading
from collections import defaultdict

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


class _Mailbox:
    def __init__(self):
        self.lock = threading.Lock()
        self.boxes = defaultdict(queue.Queue)

    def box(self, src, dst):
        with self.lock:
            return self.boxes[(src, dst)]


class _Done:
    def wait(self):
        return True


class _Recv:
    def __init__(self, box, buf):
        self.box, self.buf = box, buf

    def wait(self):
        self.buf.copy_(self.box.get(timeout=120))
        return True


class _Comm:
    """The point-to-point subset of torch.distributed over a mailbox."""
    isend, irecv = "send", "recv"

    def __init__(self, mail, world, rank):
        self.mail, self.world, self.rank = mail, world, rank

    def get_world_size(self, group=None):
        return self.world

    def get_rank(self, group=None):
        return self.rank

    def get_global_rank(self, group, rank):
        return rank

    @staticmethod
    def P2POp(op, tensor, peer, group=None):
        return (op, tensor, peer)

    def batch_isend_irecv(self, ops):
        reqs = []
        for op, t, peer in ops:
            if op == "send":
                self.mail.box(self.rank, peer).put(t.clone())
                reqs.append(_Done())
            else:
                reqs.append(_Recv(self.mail.box(peer, self.rank), t))
        return reqs


@pytest.mark.parametrize("shape,r,world,overlap", [
    ("star", 4, 2, True), ("star", 4, 3, False), ("box", 2, 2, True), ("box", 1, 3, True)])
def test_slab_sweeps_on_the_gpu_match_the_whole_grid(shape, r, world, overlap):
    import paper_2507_11067_gb300 as mms
    from paper_2507_11067_gb300 import distributed as mdist
    assert torch.cuda.is_available()
    n, steps = (150, 70, 37), 3
    grid = workloads.uniform_grid(*n, r, workload=2, salt=950 + r)
    c = workloads.normal_coeffs(shape, r, workload=2, salt=950 + r)
    dev = torch.from_numpy(grid).cuda()

    # the whole grid, iterated with the library
    whole = dev.clone()
    for _ in range(steps):
        out = mms.apply(shape, r, c, whole)
        whole[r:-r, r:-r, r:-r].copy_(out)

    mail = _Mailbox()
    results, errors = {}, []

    def rank_main(k):
        try:
            torch.cuda.set_device(0)
            ss = mdist.SlabSweep(shape, r, c, *n, comm=_Comm(mail, world, k))
            slab = ss.local_slab(dev).clone()
            res = ss.iterate(slab, steps, overlap=overlap)
            torch.cuda.synchronize()
            results[k] = (ss.z0, ss.z1, res.cpu())
        except Exception as e:      # surfaced below
            errors.append(repr(e))

    threads = [threading.Thread(target=rank_main, args=(k,)) for k in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    mms.check_device()
    assert not errors, errors
    assert sorted(results) == list(range(world))

    ref = grid.astype(np.float64)
    for _ in range(steps):
        ref[r:-r, r:-r, r:-r] = oracle.stencil(shape, r, c, ref)
    whole = whole.cpu().numpy()
    scale = np.abs(ref).max()
    for k in range(world):
        z0, z1, slab = results[k]
        part = slab.numpy()
        err_whole = np.abs(part - whole[z0:z1 + 2 * r]).max() / scale
        err_ref = np.abs(part - ref[z0:z1 + 2 * r]).max() / scale
        print(f"{shape} r={r} rank {k}/{world} planes [{z0},{z1}) overlap={overlap}: "
              f"vs whole-grid library {err_whole:.2e}, vs oracle {err_ref:.2e}")
        assert err_whole <= 1e-5 and err_ref <= 1e-5 * steps
