"""mms_stencil_apply_host: sweeps of grids in host memory, streamed through
the device in z-slabs, against the FP64 oracle (several slabs, a ragged last
slab, pinned and pageable host memory, every path)."""
import numpy as np
import pytest

import oracle
import paper_2507_11067_gb300 as mms
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"cuda_core": 1e-5, "auto": 1e-5, "bf16x3": 1e-5, "3xtf32": 1e-5, "naive": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    mms.build()
    mms.load()
    assert torch.cuda.is_available()


def rel(g, o):
    return float(np.abs(np.asarray(g, np.float64) - o).max() / max(np.abs(o).max(), 1e-300))


def host_grid(grid, r, pinned):
    Z, Y, X = grid.shape
    t = mms.padded_empty(X - 2 * r, Y - 2 * r, Z - 2 * r, r, device="cpu", zero=False)
    if pinned:
        t = torch.as_strided(torch.empty(t.untyped_storage().nbytes() // 4, pin_memory=True), t.shape, t.stride())
    t.copy_(torch.from_numpy(grid))
    return t


@pytest.mark.parametrize("shape,r,path", [("box", 1, "cuda_core"), ("box", 2, "auto"), ("box", 2, "bf16x3"),
                                          ("star", 4, "cuda_core"), ("star", 2, "3xtf32"),
                                          ("box", 3, "naive")])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_sweep_matches_oracle(shape, r, path, pinned):
    n = (45, 38, 37)   # 37 planes: slabs of 8, the last one 5 planes
    grid = workloads.uniform_grid(*n, r, workload=2, salt=90 + r)
    c = workloads.normal_coeffs(shape, r, workload=2, salt=90 + r)
    ref = oracle.stencil(shape, r, c, grid)
    hin = host_grid(grid, r, pinned)
    hout = torch.full((n[2], n[1], n[0]), float("nan"), pin_memory=pinned)
    mms.apply_host(shape, r, c, hin, hout, path=path)
    torch.cuda.synchronize()
    mms.check_device()
    err = rel(hout.numpy(), ref)
    print(f"host {shape} r={r} {path} pinned={pinned}: max-rel {err:.3e}")
    assert err <= TOL[path]
    # the input is left as it was
    assert torch.equal(hin, torch.from_numpy(grid))


def test_host_sweep_output_pitch_and_canary():
    r, n = 2, (30, 20, 19)
    grid = workloads.uniform_grid(*n, r, workload=2, salt=95)
    c = workloads.normal_coeffs("box", r, workload=2, salt=95)
    ref = oracle.stencil("box", r, c, grid)
    base = torch.full((n[2], n[1], 36), 7.25, pin_memory=True)
    out = base[:, :, :30]
    mms.apply_host("box", r, c, host_grid(grid, r, True), out, path="cuda_core")
    torch.cuda.synchronize()
    assert rel(out.numpy(), ref) <= 1e-5
    assert torch.all(base[:, :, 30:] == 7.25)
