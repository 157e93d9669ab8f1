"""GPU parity of the FP64 sweeps (mms_stencil_apply_f64) against the FP64
oracle: both sides compute the same sums in double precision, so the bar is
max|gpu - oracle| / max|oracle| <= 1e-13 (summation order only)."""
import numpy as np
import pytest

import oracle
import paper_2507_11067_gb300 as mms
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mms.build()
    mms.load()
    assert torch.cuda.is_available()


def rel(g, o):
    return float(np.abs(np.asarray(g, np.float64) - o).max() / max(np.abs(o).max(), 1e-300))


def _coeffs(shape, r, salt):
    return workloads.normal_coeffs(shape, r, workload=2, salt=salt).astype(np.float64)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("shape", ["star", "box", "star2d", "box2d"])
def test_f64_sweep_matches_oracle(shape, r):
    planar = shape in ("star2d", "box2d")
    nx, ny, nz = (70, 45, 3) if planar else (37, 29, 23)
    g = np.random.default_rng(500 + r)
    zpad = 0 if planar else 2 * r
    grid = np.zeros((nz + zpad, ny + 2 * r, nx + 2 * r))
    grid[...] = g.uniform(-1, 1, grid.shape)       # the halo carries data too
    c = _coeffs(shape, r, r)
    if planar:      # planes padded in x and y only, rows pitched to 32 doubles
        inp = torch.zeros((nz, ny + 2 * r, -(-(nx + 2 * r) // 32) * 32), device="cuda", dtype=torch.float64)
        inp = inp[..., :nx + 2 * r]
    else:
        inp = mms.padded_empty(nx, ny, nz, r, dtype=torch.float64)
    inp.copy_(torch.from_numpy(grid))
    # output with a pitch and a canary in the pad
    out_full = torch.full((nz, ny, nx + 5), 7.25, device="cuda", dtype=torch.float64)
    out = out_full[..., :nx]
    mms.apply_f64(shape, r, c, inp, out)
    torch.cuda.synchronize()
    mms.check_device()
    ref = oracle.stencil2d(shape, r, c, grid) if planar else oracle.stencil(shape, r, c, grid)
    err = rel(out.cpu().numpy(), ref)
    print(f"FP64 {shape} r={r}: {err:.2e}")
    assert err <= TOL
    assert torch.all(out_full[..., nx:] == 7.25)


def test_f64_star_512_sampled():
    n, r = 512, 4
    g = np.random.default_rng(77)
    inp = mms.padded_empty(n, n, n, r, dtype=torch.float64)
    host = np.zeros(inp.shape)
    for z in range(n + 2 * r):
        host[z, r:-r, r:-r] = g.uniform(-1, 1, (n, n)) if r <= z < n + r else 0.0
    inp.copy_(torch.from_numpy(host))
    c = workloads.fd8_star_coeffs().astype(np.float64)
    out = mms.apply_f64("star", r, c, inp)
    torch.cuda.synchronize()
    mms.check_device()
    pts = workloads.sample_points(n, n, n, 4000, workload=3)
    ref = oracle.stencil_points("star", r, c, host, pts)
    got = out.cpu().numpy()[pts[:, 2], pts[:, 1], pts[:, 0]]
    err = rel(got, ref)
    print(f"FP64 star r=4 512^3 sampled: {err:.2e}")
    assert err <= TOL


def test_f64_refuses_float32_and_tensor_core_paths():
    inp = mms.padded_empty(8, 8, 8, 1)
    with pytest.raises(ValueError):
        mms.apply_f64("star", 1, np.ones(9), inp)
