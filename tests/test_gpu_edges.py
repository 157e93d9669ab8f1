"""Degenerate and extreme shapes for the anisotropic steps and the FP64
sweeps: single planes, rows and columns, grids smaller than a tile (both the
TMA-staged TTI q pass, nx % 4 == 0, and its fallback), the maximum shot
count, and empty grids (refused by the wave-step descriptor)."""
import numpy as np
import pytest

import oracle
from oracle import aniso
import paper_2507_11067_gb300 as mms
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mms.build()
    mms.load()
    assert torch.cuda.is_available()


def rel(g, o):
    scale = max(np.abs(o).max(), 1e-300)
    return float(np.abs(np.asarray(g, np.float64) - o).max() / scale)


def _fields(n, r, nshots, k, seed):
    nx, ny, nz = n
    g = np.random.default_rng(seed)
    f = [mms.padded_empty(nx, ny, nz, r, nshots=nshots) for _ in range(k)]
    for x in f[:4]:
        x[:, r:-r, r:-r, r:-r] = torch.from_numpy(g.uniform(-1, 1, (nshots, nz, ny, nx)).astype(np.float32))
    return f


def _desc(n, r, nshots, f, src):
    py, pz, ss = mms.field_geometry(f[0])
    return mms.wave_desc(*n, r, nshots, py, pz, ss, 0, 0.0, -1, src)


SIZES = [(1, 1, 1), (3, 2, 5), (5, 9, 1), (8, 1, 3), (4, 7, 2), (70, 3, 1)]


@pytest.mark.parametrize("r", [1, 4])
@pytest.mark.parametrize("n", SIZES)
def test_vti_tiny_grids(n, r):
    nx, ny, nz = n
    g = np.random.default_rng(7)
    vp = g.uniform(1500, 3000, (nz, ny, nx)).astype(np.float32)
    eps = g.uniform(0, 0.3, (nz, ny, nx)).astype(np.float32)
    delta = g.uniform(-0.1, 0.2, (nz, ny, nx)).astype(np.float32)
    f = _fields(n, r, 1, 6, 11)
    src = [(nx - 1, ny // 2, nz - 1)]
    desc, _s = _desc(n, r, 1, f, src)
    mv, rho = mms.padded_empty(nx, ny, nz, r), mms.padded_empty(nx, ny, nz, r)
    dev = [torch.from_numpy(x).cuda() for x in (vp, eps, delta)]
    mms.vti_model(desc, *dev, mv, rho, 1e-3, 10.0)
    cf = workloads.normal_coeffs("star", r, workload=6, salt=r)
    amp = torch.full((1,), 0.75, device="cuda")
    mms.vti_step(desc, cf, mv, rho, *f[:4], f[4], f[5], amp)
    torch.cuda.synchronize()
    mms.check_device()
    host = [x[0].cpu().numpy().astype(np.float64) for x in f[:4]]
    mh, mvo = aniso.vti_medium(vp, eps, delta, 1e-3, 10.0)
    oh, ov = aniso.vti_step(r, cf, mh, mvo, None, src[0], 0.75, *host)
    assert rel(f[4][0].cpu().numpy(), oh) <= TOL and rel(f[5][0].cpu().numpy(), ov) <= TOL


@pytest.mark.parametrize("r", [1, 4])
@pytest.mark.parametrize("n", SIZES)
def test_tti_tiny_grids(n, r):
    nx, ny, nz = n
    g = np.random.default_rng(8)
    shp = (nz, ny, nx)
    ins = [g.uniform(1500, 3000, shp), g.uniform(500, 1000, shp), g.uniform(0, 0.3, shp),
           g.uniform(-0.1, 0.2, shp), g.uniform(0.7, 1.3, shp), g.uniform(0, np.pi / 2, shp),
           g.uniform(-np.pi, np.pi, shp)]
    ins = [x.astype(np.float32) for x in ins]
    f = _fields(n, r, 1, 6, 12)
    src = [(0, 0, 0)]
    desc, _s = _desc(n, r, 1, f, src)
    med = torch.empty((8,) + shp, device="cuda")
    mms.tti_model(desc, *[torch.from_numpy(x).cuda() for x in ins], med, 1e-3, 10.0)
    work = torch.empty((4, 1) + shp, device="cuda")
    w2, w1 = aniso.fd2_row(r).astype(np.float32), aniso.fd1_row(r).astype(np.float32)
    amp = torch.full((1,), 0.5, device="cuda")
    mms.tti_step(desc, w2, w1, med, *f[:4], f[4], f[5], work, amp)
    torch.cuda.synchronize()
    mms.check_device()
    host = [x[0].cpu().numpy().astype(np.float64) for x in f[:4]]
    vp, vs, eps, delta, al, th, ph = ins
    op, oq = aniso.tti_step(r, aniso.tti_medium(vp, vs, eps, delta, al, 1e-3, 10.0), aniso.tilt_axis(th, ph),
                            None, src[0], 0.5, *host, w2, w1)
    assert rel(f[4][0].cpu().numpy(), op) <= TOL and rel(f[5][0].cpu().numpy(), oq) <= TOL


def test_vti_64_shots():
    # the maximum shot count of the descriptor, each shot its own source
    n, r, ns = (12, 10, 9), 4, 64
    nx, ny, nz = n
    f = _fields(n, r, ns, 6, 13)
    g = np.random.default_rng(14)
    src = [(int(g.integers(nx)), int(g.integers(ny)), int(g.integers(nz))) for _ in range(ns)]
    desc, _s = _desc(n, r, ns, f, src)
    vp = np.full((nz, ny, nx), 2000.0, np.float32)
    eps = np.full_like(vp, 0.2)
    delta = np.full_like(vp, 0.1)
    mv, rho = mms.padded_empty(nx, ny, nz, r), mms.padded_empty(nx, ny, nz, r)
    mms.vti_model(desc, *[torch.from_numpy(x).cuda() for x in (vp, eps, delta)], mv, rho, 1e-3, 10.0)
    cf = workloads.fd8_star_coeffs()
    amps = torch.linspace(0.1, 6.4, ns, device="cuda")
    mms.vti_step(desc, cf, mv, rho, *f[:4], f[4], f[5], amps)
    torch.cuda.synchronize()
    mms.check_device()
    mh, mvo = aniso.vti_medium(vp, eps, delta, 1e-3, 10.0)
    for s in (0, 17, 63):
        host = [x[s].cpu().numpy().astype(np.float64) for x in f[:4]]
        oh, ov = aniso.vti_step(r, cf, mh, mvo, None, src[s], float(amps[s]), *host)
        assert rel(f[4][s].cpu().numpy(), oh) <= TOL and rel(f[5][s].cpu().numpy(), ov) <= TOL
    d65, _ = mms.wave_desc(nx, ny, nz, r, 65, *mms.field_geometry(f[0]), 0, 0.0, -1, None)
    with pytest.raises(mms.MMSError):
        mms.vti_step(d65, cf, mv, rho, *f[:4], f[4], f[5], amps)


def test_empty_wave_grids_are_refused():
    f = _fields((4, 4, 4), 1, 1, 6, 15)
    d0, _ = mms.wave_desc(0, 4, 4, 1, 1, *mms.field_geometry(f[0]), 0, 0.0, -1, None)
    mv = mms.padded_empty(4, 4, 4, 1)
    with pytest.raises(mms.MMSError):
        mms.vti_step(d0, np.ones(9), mv, mv, *f[:4], f[4], f[5], torch.zeros(1, device="cuda"))


@pytest.mark.parametrize("shape", ["star", "box"])
@pytest.mark.parametrize("n", [(1, 1, 1), (2, 3, 1), (1, 5, 7)])
def test_f64_tiny_grids(shape, n):
    r = 2
    nx, ny, nz = n
    g = np.random.default_rng(16)
    grid = g.uniform(-1, 1, (nz + 2 * r, ny + 2 * r, nx + 2 * r))
    inp = mms.padded_empty(nx, ny, nz, r, dtype=torch.float64)
    inp.copy_(torch.from_numpy(grid))
    c = workloads.normal_coeffs(shape, r, workload=2).astype(np.float64)
    out = mms.apply_f64(shape, r, c, inp)
    torch.cuda.synchronize()
    mms.check_device()
    assert rel(out.cpu().numpy(), oracle.stencil(shape, r, c, grid)) <= 1e-13
