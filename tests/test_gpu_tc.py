"""GPU parity of the tensor-core (tcgen05) banded box sweeps against the oracle.

Split-precision paths (3xTF32, BF16x3: hi*hi + hi*lo + lo*hi, FP32
accumulation) meet the FP32 bar max|gpu - oracle| / max|oracle| <= 1e-5;
the single-product TF32 path is reported and held to a TF32-level bound.
"""
import numpy as np
import pytest

import oracle
import paper_2507_11067_gb300 as mms
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"3xtf32": 1e-5, "bf16x3": 1e-5, "tf32": 5e-3}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mms.build()
    mms.load()
    assert torch.cuda.is_available()


def rel(g, o):
    return float(np.abs(np.asarray(g, np.float64) - o).max() / max(np.abs(o).max(), 1e-300))


# ragged tiles in x and y; z chunks of 64, 32, 128, 16, 52 or 40 planes
# (the variants) leave one-plane and ragged last chunks (nz = 1, 17, 37)
SIZES = [(53, 41, 19), (24, 28, 8), (7, 5, 3), (100, 70, 37), (40, 35, 1), (33, 29, 17)]


@pytest.mark.parametrize("path", ["bf16x3", "3xtf32", "tf32"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_box_tc_matches_oracle(path, r):
    if mms.num_variants("box", r, path) == 0:
        with pytest.raises(mms.MMSError, match="UNSUPPORTED"):
            grid = workloads.uniform_grid(8, 8, 8, r, workload=2)
            mms.apply("box", r, np.ones((2 * r + 1) ** 3, np.float32), mms.to_padded_device(grid, r),
                      path=path)
        return
    for k, n in enumerate(SIZES):
        grid = workloads.uniform_grid(*n, r, workload=2, salt=300 + 10 * r + k)
        c = workloads.normal_coeffs("box", r, workload=2, salt=300 + 10 * r + k)
        ref = oracle.stencil("box", r, c, grid)
        inp = mms.to_padded_device(grid, r)
        for v in range(mms.num_variants("box", r, path)):
            out = mms.apply("box", r, c, inp, path=path, variant=v)
            torch.cuda.synchronize()
            mms.check_device()
            err = rel(out.cpu().numpy(), ref)
            print(f"box r={r} {path} n={n} variant={v}: max-rel error {err:.3e}")
            assert err <= TOL[path], (n, v, err)


@pytest.mark.parametrize("path", ["bf16x3", "3xtf32"])
def test_box_tc_512_sampled(path):
    # Full 512^3 box r=2 (125 points) in the launch configuration the
    # benchmark times (the default / tuned variant).
    r, n = 2, 512
    if mms.num_variants("box", r, path) == 0:
        pytest.skip("path not built for r=2")
    grid = workloads.uniform_grid(n, n, n, r, workload=2, salt=r)
    c = workloads.normal_coeffs("box", r, workload=2, salt=r)
    pts = workloads.sample_points(n, n, n, 3000, workload=2)
    ref = oracle.stencil_points("box", r, c, grid, pts)
    inp = mms.to_padded_device(grid, r)
    del grid
    out = mms.apply("box", r, c, inp, path=path)
    torch.cuda.synchronize()
    mms.check_device()
    got = out[pts[:, 2], pts[:, 1], pts[:, 0]].cpu().numpy()
    err = rel(got, ref)
    print(f"box r=2 512^3 {path}: sampled max-rel error {err:.3e}")
    assert err <= TOL[path]
    # the tensor-core result agrees with the CUDA-core sweep everywhere
    cc = mms.apply("box", r, c, inp, path="cuda_core")
    torch.cuda.synchronize()
    diff = (out - cc).abs().max().item() / cc.abs().max().item()
    assert diff <= 2 * TOL[path]


@pytest.mark.parametrize("r", [1, 2])
def test_box_tc_many_tiles_per_cta(r):
    # More tiles than resident CTAs, so that each persistent CTA runs
    # several tiles in a row and its two mixed workers (box r = 1, 2 on two
    # CTAs per SM) carry their plane and output cursors across tile ends;
    # the last z chunk has an odd number of output planes (603 = 37 x 16 +
    # 11 = 15 x 40 + 3); 400 to 1140 tiles for 304 CTAs.  Every point
    # against the oracle.
    n = (200, 150, 603)
    grid = workloads.uniform_grid(*n, r, workload=2, salt=40 + r)
    c = workloads.normal_coeffs("box", r, workload=2, salt=40 + r)
    ref = oracle.stencil("box", r, c, grid)
    inp = mms.to_padded_device(grid, r)
    for v in (3, 5):   # 16- and 40-plane z chunks
        out = mms.apply("box", r, c, inp, path="bf16x3", variant=v)
        torch.cuda.synchronize()
        mms.check_device()
        err = rel(out.cpu().numpy(), ref)
        print(f"box r={r} bf16x3 {n} variant {v}: max-rel error {err:.3e}")
        assert err <= TOL["bf16x3"], (v, err)


def test_every_tensor_core_combination_is_built():
    for shape in ("box", "star"):
        for path in ("bf16x3", "3xtf32", "tf32"):
            for r in (1, 2, 3, 4):
                assert mms.num_variants(shape, r, path) > 0, (shape, path, r)


@pytest.mark.parametrize("path", ["bf16x3", "3xtf32", "tf32"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_star_tc_matches_oracle(path, r):
    # Star on tensor cores, every variant: the single-pass form (x/y lines
    # and centre as a planar band, z line summed by the converter warps) and
    # the paper's two-pass form (planar pass into a temporary grid, then the
    # z part on CUDA cores).
    nvar = mms.num_variants("star", r, path)
    assert nvar > 0
    for k, n in enumerate([(53, 41, 19), (30, 66, 9), (40, 35, 1), (33, 29, 17)]):
        grid = workloads.uniform_grid(*n, r, workload=3, salt=500 + 10 * r + k)
        c = workloads.star_coeffs(r) if r == 4 else workloads.normal_coeffs("star", r, workload=3, salt=k)
        ref = oracle.stencil("star", r, c, grid)
        inp = mms.to_padded_device(grid, r)
        for v in range(nvar):
            out = mms.apply("star", r, c, inp, path=path, variant=v)
            torch.cuda.synchronize()
            mms.check_device()
            err = rel(out.cpu().numpy(), ref)
            print(f"star r={r} {path} n={n} variant={v}: max-rel error {err:.3e}")
            assert err <= TOL[path], (n, v, err)
