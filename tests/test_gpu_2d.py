"""GPU parity of the planar stencils (Table I's 2D kernels, star2d and box2d)
against the oracle: every path and tile variant on grids with several tiles
and ragged edges (batches of planes and single planes), the 8192^2 plane at
sampled points in the benchmark's launch configuration, and the host-memory
entry point."""
import numpy as np
import pytest

import oracle
import paper_2507_11067_gb300 as mms
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"naive": 1e-5, "cuda_core": 1e-5, "auto": 1e-5, "bf16x3": 1e-5, "3xtf32": 1e-5, "tf32": 5e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    mms.build()
    mms.load()
    assert torch.cuda.is_available()


def rel(g, o):
    return float(np.abs(np.asarray(g, np.float64) - o).max() / max(np.abs(o).max(), 1e-300))


SIZES = [(75, 53, 3), (130, 97, 1), (9, 5, 2)]


@pytest.mark.parametrize("shape", ["star2d", "box2d"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_planar_every_path_matches_oracle(shape, r):
    for k, n in enumerate(SIZES):
        grid = workloads.uniform_grid2d(*n, r, workload=6, salt=10 * r + k)
        c = workloads.normal_coeffs(shape, r, workload=6, salt=10 * r + k)
        ref = oracle.stencil2d(shape, r, c, grid)
        inp = mms.to_padded_device2d(grid, r)
        for path in ("naive", "cuda_core", "bf16x3", "3xtf32", "tf32"):
            nv = mms.num_variants(shape, r, path)
            assert nv > 0, (shape, r, path)
            for v in (range(nv) if path == "cuda_core" else (0, nv - 1)):
                out = mms.apply(shape, r, c, inp, path=path, variant=v)
                torch.cuda.synchronize()
                mms.check_device()
                err = rel(out.cpu().numpy(), ref)
                assert err <= TOL[path], (n, path, v, err)


@pytest.mark.parametrize("shape,r", [("star2d", 2), ("star2d", 4), ("box2d", 2), ("box2d", 3)])
def test_table1_2d_kernels_8192_sampled(shape, r):
    # Table I's 2D kernels on one 8192^2 plane, AUTO with the tuned table
    from paper_2507_11067_gb300 import tune
    chosen = tune.load_table()
    try:
        n = 8192
        grid = workloads.uniform_grid2d(n, n, 1, r, workload=6, salt=r)
        c = workloads.normal_coeffs(shape, r, workload=6, salt=r)
        g = workloads.rng(6, 99)
        pts = np.stack([g.integers(0, n, 3000), g.integers(0, n, 3000), np.zeros(3000, np.int64)], axis=1)
        pts = np.concatenate([pts, [[0, 0, 0], [n - 1, n - 1, 0], [0, n - 1, 0], [n - 1, 0, 0]]])
        ref = oracle.stencil2d_points(shape, r, c, grid, pts)
        inp = mms.to_padded_device2d(grid, r)
        del grid
        out = mms.apply(shape, r, c, inp, path="auto")
        torch.cuda.synchronize()
        mms.check_device()
        got = out[pts[:, 2], pts[:, 1], pts[:, 0]].cpu().numpy()
        err = rel(got, ref)
        print(f"{shape} r={r} 8192^2 ({mms.auto_path(shape, r)}): sampled max-rel {err:.3e}")
        assert err <= 1e-5
    finally:
        for key in chosen:
            mms.set_variant(*key, -1)


@pytest.mark.parametrize("shape", ["star2d", "box2d"])
def test_planar_host_sweep(shape):
    r, n = 3, (70, 45, 19)
    grid = workloads.uniform_grid2d(*n, r, workload=6, salt=50)
    c = workloads.normal_coeffs(shape, r, workload=6, salt=50)
    ref = oracle.stencil2d(shape, r, c, grid)
    hin = torch.from_numpy(grid).pin_memory()
    hout = torch.full((n[2], n[1], n[0]), float("nan"), pin_memory=True)
    mms.apply_host(shape, r, c, hin, hout, path="cuda_core")
    torch.cuda.synchronize()
    mms.check_device()
    assert rel(hout.numpy(), ref) <= 1e-5
