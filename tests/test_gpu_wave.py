"""GPU parity of the fused wave step and its adjoint against the FP64 oracle.

Teacher-forced: the oracle takes the GPU's FP32 state and does one FP64
step; the bar is max|gpu - oracle| / max|oracle| <= 1e-5.  The adjoint is
also checked against the GPU forward by dot-product tests (FP64 inner
products), which bind its transpose structure independently of the oracle.
"""
import numpy as np
import pytest

import oracle
import paper_2507_11067_gb300 as mms
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
R = 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mms.build()
    mms.load()
    assert torch.cuda.is_available()


def rel(g, o):
    return float(np.abs(np.asarray(g, np.float64) - o).max() / max(np.abs(o).max(), 1e-300))


class Setup:
    def __init__(self, nx=45, ny=38, nz=41, nshots=3, nsteps=30, sponge=6, seed=0):
        self.nx, self.ny, self.nz, self.ns = nx, ny, nz, nshots
        self.w = workloads.WaveInputs(nx, ny, nz, nshots=nshots, nsteps=nsteps, sponge=sponge,
                                      salt=seed)
        self.cf = workloads.fd8_star_coeffs()
        self.m = mms.padded_empty(nx, ny, nz, R)
        self.fields = [mms.padded_empty(nx, ny, nz, R, nshots=nshots) for _ in range(4)]
        py, pz, ss = mms.field_geometry(self.fields[0])
        self.desc, self._src = mms.wave_desc(nx, ny, nz, R, nshots, py, pz, ss, self.w.sponge,
                                             self.w.sponge_a, self.w.zrec, self.w.src)
        self.v = torch.from_numpy(self.w.v).cuda()
        mms.model_from_velocity(self.desc, self.v, self.m, self.w.dt, self.w.h)
        self.amps = torch.from_numpy(self.w.amp).cuda().contiguous()
        self.prob = oracle.WaveProblem(R, self.cf, oracle.model_m(self.w.v, self.w.dt, self.w.h),
                                       (self.w.sponge, self.w.sponge_a), self.w.src, self.w.amp,
                                       self.w.zrec)

    def fill(self, f, seed):
        g = np.random.default_rng(seed)
        f[:, R:-R, R:-R, R:-R] = torch.from_numpy(
            g.uniform(-1, 1, (self.ns, self.nz, self.ny, self.nx)).astype(np.float32))

    def host(self, f):
        return f.cpu().numpy().astype(np.float64)


def test_model_from_velocity():
    s = Setup()
    m = s.m.cpu().numpy()
    ref = oracle.model_m(s.w.v, s.w.dt, s.w.h)
    assert rel(m[R:-R, R:-R, R:-R], ref) <= 1e-6
    assert np.all(m[:R] == 0) and np.all(m[:, :, :R] == 0)


def test_teacher_forced_step():
    s = Setup()
    cur, prev = s.fields[0], s.fields[1]
    s.fill(cur, 1)
    s.fill(prev, 2)
    c0, p0 = s.host(cur), s.host(prev)
    rec = torch.zeros((s.ns, s.ny, s.nx), device="cuda")
    n = 3
    mms.wave_step(s.desc, s.cf, s.m, cur, prev, s.amps[n], rec)
    torch.cuda.synchronize()
    mms.check_device()
    got = prev.cpu().numpy()
    for sh in range(s.ns):
        ref = s.prob.step(c0[sh], p0[sh], sh, n)
        assert rel(got[sh], ref) <= TOL
        assert np.array_equal(rec[sh].cpu().numpy(), got[sh, R + s.w.zrec, R:-R, R:-R])
        # the zero halo is never written
        assert np.all(got[sh, :R] == 0) and np.all(got[sh, :, :, -R:] == 0)


def test_source_only_step_is_exact_at_source():
    # From zero states the first step is G s at the source point only.
    s = Setup(nshots=2)
    cur, prev = s.fields[0], s.fields[1]
    amp = torch.tensor([0.5, -2.0], device="cuda")
    mms.wave_step(s.desc, s.cf, s.m, cur, prev, amp)
    torch.cuda.synchronize()
    got = prev.cpu().numpy()
    for sh, (x, y, z) in enumerate(s.w.src):
        nz_idx = np.argwhere(got[sh] != 0)
        assert len(nz_idx) == 1 and tuple(nz_idx[0]) == (z + R, y + R, x + R)
        g = s.prob.gx[x] * s.prob.gy[y] * s.prob.gz[z]
        assert got[sh, z + R, y + R, x + R] == pytest.approx(g * amp[sh].item(), rel=1e-6)


def test_trajectory_against_oracle():
    # 60 steps from rest: FP32 drift against the FP64 oracle stays small.
    nsteps = 60
    s = Setup(nshots=2, nsteps=nsteps)
    rec = torch.zeros((nsteps, s.ns, s.ny, s.nx), device="cuda")
    mms.wave_forward(s.desc, s.cf, s.m, s.amps, nsteps, s.fields[0], s.fields[1], rec)
    torch.cuda.synchronize()
    mms.check_device()
    ref, _ = s.prob.forward(nsteps)
    err = rel(rec.cpu().numpy(), ref)
    assert err <= 1e-4, err


def _flat(f):
    """The whole storage of a (pitched) field view, as one flat float view."""
    return torch.as_strided(f, (f.untyped_storage().nbytes() // 4,), (1,), 0)


def test_forward_graph_matches_steps_and_checkpoints():
    nsteps, every = 25, 10
    s = Setup(nshots=2, nsteps=nsteps)
    a0, a1, b0, b1 = s.fields
    rec_a = torch.zeros((nsteps, s.ns, s.ny, s.nx), device="cuda")
    rec_b = torch.zeros_like(rec_a)
    fb = a0.untyped_storage().nbytes() // 4
    ckpt = torch.zeros((3, 2, fb), device="cuda")
    saved = {}
    for k in range(nsteps):
        cur, prev = (a1, a0) if k % 2 == 0 else (a0, a1)
        if k % every == 0:
            saved[k // every] = (_flat(cur).clone(), _flat(prev).clone())
        mms.wave_step(s.desc, s.cf, s.m, cur, prev, s.amps[k], rec_a[k])
    mms.wave_forward(s.desc, s.cf, s.m, s.amps, nsteps, b0, b1, rec_b, ckpt, every, graph=True)
    torch.cuda.synchronize()
    mms.check_device()
    assert torch.equal(rec_a, rec_b)
    assert torch.equal(a0, b0) and torch.equal(a1, b1)
    for j in range(3):   # checkpoint j holds (a^{10 j}, a^{10 j - 1})
        assert torch.equal(ckpt[j, 0], saved[j][0]) and torch.equal(ckpt[j, 1], saved[j][1])
    # a replay of the cached graph gives the same records again
    rec_b.zero_()
    b0.zero_()
    b1.zero_()
    mms.wave_forward(s.desc, s.cf, s.m, s.amps, nsteps, b0, b1, rec_b, ckpt, every, graph=True)
    torch.cuda.synchronize()
    assert torch.equal(rec_a, rec_b)


def test_teacher_forced_adjoint_step():
    s = Setup(nshots=2)
    lam1, lam2, a_n = s.fields[0], s.fields[1], s.fields[2]
    for f, sd in ((lam1, 3), (lam2, 4), (a_n, 5)):
        s.fill(f, sd)
    l1, l2, an = s.host(lam1), s.host(lam2), s.host(a_n)
    g = np.random.default_rng(9)
    resid = torch.from_numpy(g.normal(size=(s.ns, s.ny, s.nx)).astype(np.float32)).cuda()
    grad = torch.zeros((s.nz, s.ny, s.nx), device="cuda", dtype=torch.float64)
    mms.wave_adjoint(s.desc, s.cf, s.m, lam1, lam2, resid, a_n, grad)
    torch.cuda.synchronize()
    mms.check_device()
    got = lam2.cpu().numpy()
    gref = np.zeros((s.nz, s.ny, s.nx))
    rh = resid.cpu().numpy().astype(np.float64)
    for sh in range(s.ns):
        ref = s.prob.adjoint_step(l1[sh], l2[sh], rh[sh], an[sh], gref)
        assert rel(got[sh], ref) <= TOL
    assert rel(grad.cpu().numpy(), gref) <= TOL


def test_grad256_adjoint_step_full_size():
    # the gradient workload's size and launch (2 shots x 256^3, 20-cell
    # sponge, receivers on the first non-sponge plane): one teacher-forced
    # adjoint step with its FP64 gradient term, every point against the oracle
    s = Setup(nx=256, ny=256, nz=256, nshots=2, nsteps=4, sponge=20, seed=3)
    lam1, lam2, a_n = s.fields[0], s.fields[1], s.fields[2]
    for f, sd in ((lam1, 31), (lam2, 32), (a_n, 33)):
        s.fill(f, sd)
    l1, l2, an = s.host(lam1), s.host(lam2), s.host(a_n)
    g = np.random.default_rng(34)
    resid = torch.from_numpy(g.normal(size=(s.ns, s.ny, s.nx)).astype(np.float32)).cuda()
    grad = torch.zeros((s.nz, s.ny, s.nx), device="cuda", dtype=torch.float64)
    mms.wave_adjoint(s.desc, s.cf, s.m, lam1, lam2, resid, a_n, grad)
    torch.cuda.synchronize()
    mms.check_device()
    got = lam2.cpu().numpy()
    gref = np.zeros((s.nz, s.ny, s.nx))
    rh = resid.cpu().numpy().astype(np.float64)
    for sh in range(s.ns):
        ref = s.prob.adjoint_step(l1[sh], l2[sh], rh[sh], an[sh], gref)
        e = rel(got[sh], ref)
        print(f"adjoint step 256^3 shot {sh}: {e:.2e}")
        assert e <= TOL
    e = rel(grad.cpu().numpy(), gref)
    print(f"gradient term 256^3: {e:.2e}")
    assert e <= TOL


def test_step_lap_and_adjoint_lap():
    # mms_wave_step_lap: the same a^{n+1} as mms_wave_step_to, plus L a^n;
    # mms_wave_adjoint_lap fed that L a^n: the same lam^n as mms_wave_adjoint
    # fed a^n, and the same gradient up to the summation order of L a^n
    s = Setup(nshots=2)
    cur, prev, nxt, lap = s.fields
    s.fill(cur, 41)
    s.fill(prev, 42)
    ref_next = mms.padded_empty(s.nx, s.ny, s.nz, R, nshots=2)
    mms.wave_step_to(s.desc, s.cf, s.m, cur, prev, ref_next, s.amps[2])
    mms.wave_step_lap(s.desc, s.cf, s.m, cur, prev, nxt, lap, s.amps[2])
    torch.cuda.synchronize()
    mms.check_device()
    assert torch.equal(nxt, ref_next)
    c = s.host(cur)
    for sh in range(2):
        ref = oracle.stencil("star", R, s.cf, c[sh])
        assert rel(lap[sh, R:-R, R:-R, R:-R].cpu().numpy(), ref) <= TOL
    lam1 = mms.padded_empty(s.nx, s.ny, s.nz, R, nshots=2)
    s.fill(lam1, 43)
    g = np.random.default_rng(44)
    resid = torch.from_numpy(g.normal(size=(2, s.ny, s.nx)).astype(np.float32)).cuda()
    out = []
    for fn, a in ((mms.wave_adjoint, cur), (mms.wave_adjoint_lap, lap)):
        lam2 = mms.padded_empty(s.nx, s.ny, s.nz, R, nshots=2)
        s.fill(lam2, 45)
        grad = torch.zeros((s.nz, s.ny, s.nx), device="cuda", dtype=torch.float64)
        fn(s.desc, s.cf, s.m, lam1, lam2, resid, a, grad)
        torch.cuda.synchronize()
        mms.check_device()
        out.append((lam2.clone(), grad.cpu().numpy()))
    assert torch.equal(out[0][0], out[1][0])
    assert rel(out[1][1], out[0][1]) <= 1e-6
    # no gradient term without L a^n
    lam2 = mms.padded_empty(s.nx, s.ny, s.nz, R, nshots=2)
    s.fill(lam2, 45)
    grad = torch.zeros((s.nz, s.ny, s.nx), device="cuda", dtype=torch.float64)
    mms.wave_adjoint_lap(s.desc, s.cf, s.m, lam1, lam2, resid, None, grad)
    torch.cuda.synchronize()
    assert torch.equal(lam2, out[0][0]) and float(grad.abs().max()) == 0.0
    with pytest.raises(mms.MMSError):
        mms.wave_step_lap(s.desc, s.cf, s.m, cur, prev, nxt, cur, s.amps[2])   # L a^n over a^n


def test_out_of_place_step_matches_in_place_step():
    s = Setup(nshots=2)
    cur, prev, work, nxt = s.fields
    s.fill(cur, 21)
    s.fill(prev, 22)
    work.copy_(prev)
    before = prev.clone()
    mms.wave_step(s.desc, s.cf, s.m, cur, work, s.amps[3])
    mms.wave_step_to(s.desc, s.cf, s.m, cur, prev, nxt, s.amps[3])
    torch.cuda.synchronize()
    mms.check_device()
    assert torch.equal(nxt, work)            # the same arithmetic, bit for bit
    assert torch.equal(prev, before)         # a^{n-1} is only read
    assert not nxt[:, :R].any() and not nxt[:, -R:].any()   # the halo is not written


def test_adjoint_per_shot_gradient_slices():
    s = Setup(nshots=3)
    lam1, lam2, a_n, lam2b = s.fields
    for f, sd in ((lam1, 31), (lam2, 32), (a_n, 33)):
        s.fill(f, sd)
    lam2b.copy_(lam2)
    l1, l2, an = s.host(lam1), s.host(lam2), s.host(a_n)
    g = np.random.default_rng(34)
    resid = torch.from_numpy(g.normal(size=(s.ns, s.ny, s.nx)).astype(np.float32)).cuda()
    shared = torch.zeros((s.nz, s.ny, s.nx), device="cuda", dtype=torch.float64)
    mms.wave_adjoint(s.desc, s.cf, s.m, lam1, lam2, resid, a_n, shared)
    npts = s.nz * s.ny * s.nx
    py, pz, ss = mms.field_geometry(lam1)
    desc_g, _keep = mms.wave_desc(s.nx, s.ny, s.nz, R, s.ns, py, pz, ss, s.w.sponge, s.w.sponge_a,
                                  s.w.zrec, s.w.src, grad_shot_stride=npts)
    slices = torch.full((s.ns, s.nz, s.ny, s.nx), 0.25, device="cuda", dtype=torch.float64)
    mms.wave_adjoint(desc_g, s.cf, s.m, lam1, lam2b, resid, a_n, slices)
    torch.cuda.synchronize()
    mms.check_device()
    assert torch.equal(lam2, lam2b)          # lam^n does not depend on the gradient layout
    rh = resid.cpu().numpy().astype(np.float64)
    for sh in range(s.ns):
        gref = np.full((s.nz, s.ny, s.nx), 0.25)   # accumulated onto what was there
        s.prob.adjoint_step(l1[sh], l2[sh], rh[sh], an[sh], gref)
        assert rel(slices[sh].cpu().numpy(), gref) <= TOL
    total = mms.sum_f64(slices, slices[0]).cpu().numpy() - 0.25 * s.ns
    assert np.abs(total - shared.cpu().numpy()).max() <= 1e-12 * np.abs(total).max()


def _dot(a, b):
    out = torch.zeros(1, device="cuda", dtype=torch.float64)
    mms.dot_f64(a, b, out)
    return out.item()


def test_gpu_dot_product_one_step():
    # <T(u, w), lam> = <u, (2 + L m) G lam> + <w, -G^2 lam>, all on the GPU.
    s = Setup(nshots=1)
    u, w, lam, t = s.fields
    for f, sd in ((u, 11), (w, 12), (lam, 13)):
        s.fill(f, sd)
    t.copy_(w)
    mms.wave_step(s.desc, s.cf, s.m, u, t, torch.zeros(1, device="cuda"))   # t = T(u, w)
    zero = mms.padded_empty(s.nx, s.ny, s.nz, R, nshots=1)
    tu = mms.padded_empty(s.nx, s.ny, s.nz, R, nshots=1)
    mms.wave_adjoint(s.desc, s.cf, s.m, lam, tu)          # lam^{n+2} = 0: (2 + L m) G lam
    tw = mms.padded_empty(s.nx, s.ny, s.nz, R, nshots=1)
    tw.copy_(lam)
    mms.wave_adjoint(s.desc, s.cf, s.m, zero, tw)         # lam^{n+1} = 0: -G^2 lam
    torch.cuda.synchronize()
    lhs = _dot(_flat(t), _flat(lam))
    rhs = _dot(_flat(u), _flat(tu)) + _dot(_flat(w), _flat(tw))
    assert abs(lhs - rhs) <= 1e-6 * (abs(lhs) + abs(rhs))


# ------------------------------------------------------------ gradient
from paper_2507_11067_gb300.wave import WaveFunction, WavePropagator  # noqa: E402


def _grad_problem(n=48, nshots=2, nsteps=200, sponge=6, seed=5):
    w_true = workloads.WaveInputs(n, n, n, nshots=nshots, nsteps=nsteps, workload=5, sponge=sponge,
                                  noise=True, salt=seed)
    w0 = workloads.WaveInputs(n, n, n, nshots=nshots, nsteps=nsteps, workload=5, sponge=sponge,
                              noise=False, salt=seed)
    # same dt for both models (dt is held fixed while differentiating)
    return w_true, w0


def test_gradient_matches_oracle_48cubed():
    # 48^3 copy of the gradient workload: 2 shots, 200 steps, checkpoint every
    # 20; GPU (FP32 propagation, FP64 accumulation) vs oracle (FP64).
    w_true, w0 = _grad_problem()
    n, nsteps = 48, 200
    cf = workloads.fd8_star_coeffs()
    prop = WavePropagator(n, n, n, w0.src, w0.zrec, w0.h, w_true.dt, sponge_width=w0.sponge,
                          sponge_a=w0.sponge_a)
    amps = torch.from_numpy(w_true.amp).cuda()
    v_true = torch.from_numpy(w_true.v).cuda()
    with torch.no_grad():
        obs = WaveFunction.apply(v_true, prop, amps, nsteps, 20)
    v = torch.from_numpy(w0.v).cuda().requires_grad_(True)
    rec = WaveFunction.apply(v, prop, amps, nsteps, 20)
    loss = 0.5 * ((rec - obs) ** 2).sum()
    loss.backward()
    g_gpu = v.grad.double().cpu().numpy()
    # oracle on the same inputs
    po = oracle.WaveProblem(R, cf, oracle.model_m(w_true.v, w_true.dt, w_true.h), (w0.sponge, w0.sponge_a),
                            w0.src, w_true.amp, w0.zrec)
    obs_o, _ = po.forward(nsteps)
    p0 = oracle.WaveProblem(R, cf, oracle.model_m(w0.v, w_true.dt, w0.h), (w0.sponge, w0.sponge_a),
                            w0.src, w_true.amp, w0.zrec)
    rec_o, states = p0.forward(nsteps, keep_states=True)
    gm = p0.gradient_m(rec_o - obs_o, states)
    g_ref = gm * 2.0 * w0.v.astype(np.float64) * w_true.dt ** 2 / w0.h ** 2
    err = rel(g_gpu, g_ref)
    print(f"48^3 gradient vs oracle: max-rel {err:.3e}")
    assert err <= 1e-4
    assert rel(rec.detach().cpu().numpy(), rec_o) <= 1e-4


def test_deterministic_gradient_is_reproducible_and_matches():
    # per-shot FP64 slices: the same bits on every run, and the atomic
    # (shared-slice) gradient up to FP64 summation order
    w_true, w0 = _grad_problem(nsteps=60)
    n, nsteps = 48, 60
    prop = WavePropagator(n, n, n, w0.src, w0.zrec, w0.h, w_true.dt, sponge_width=w0.sponge,
                          sponge_a=w0.sponge_a)
    amps = torch.from_numpy(w_true.amp[:nsteps]).cuda()
    rec, ckpt = prop.forward(torch.from_numpy(w0.v).cuda(), amps, nsteps, ckpt_every=20)
    resid = (rec * 0.5).contiguous()
    g_a = prop.gradient_m(amps, resid, ckpt, 20).clone()
    g_d1 = prop.gradient_m(amps, resid, ckpt, 20, deterministic=True).clone()
    g_d2 = prop.gradient_m(amps, resid, ckpt, 20, deterministic=True).clone()
    torch.cuda.synchronize()
    mms.check_device()
    assert torch.equal(g_d1, g_d2)
    assert (g_d1 - g_a).abs().max().item() <= 1e-12 * g_a.abs().max().item()


def test_gradient_finite_difference_directions():
    # Central differences of J(v) along seeded smooth directions (GPU, FP32
    # propagation: J-cancellation limits the agreement to ~1e-2).
    w_true, w0 = _grad_problem(n=40, nsteps=120, seed=7)
    n, nsteps = 40, 120
    prop = WavePropagator(n, n, n, w0.src, w0.zrec, w0.h, w_true.dt, sponge_width=w0.sponge,
                          sponge_a=w0.sponge_a)
    amps = torch.from_numpy(w_true.amp).cuda()
    with torch.no_grad():
        obs = WaveFunction.apply(torch.from_numpy(w_true.v).cuda(), prop, amps, nsteps, 20)
    v0 = torch.from_numpy(w0.v).cuda()
    v = v0.clone().requires_grad_(True)
    J = lambda vv: float(0.5 * ((WaveFunction.apply(vv, prop, amps, nsteps, 20) - obs).double() ** 2).sum())  # noqa: E731
    loss = 0.5 * ((WaveFunction.apply(v, prop, amps, nsteps, 20) - obs) ** 2).sum()
    loss.backward()
    g = v.grad.double()
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(3)
    for _ in range(4):
        d = gaussian_filter(rng.standard_normal((n, n, n)), 4.0)
        d = torch.from_numpy(d / np.abs(d).max() * 30.0).float().cuda()   # +-30 m/s
        eps = 1.0
        with torch.no_grad():
            fd = (J(v0 + eps * d) - J(v0 - eps * d)) / (2 * eps)
        an = float((g * d.double()).sum())
        assert abs(fd - an) <= 1e-2 * abs(an), (fd, an)


def test_gpu_adjoint_dot_product_full_map():
    # Source series s -> records d is linear (d = F s); F^T r is read from
    # the adjoint states at the source: (F^T r)^n = g_src lam^{n+1}[src].
    nsteps = 60
    s = Setup(nshots=1, nsteps=nsteps)
    g = np.random.default_rng(21)
    amps = torch.from_numpy(g.normal(size=(nsteps, 1)).astype(np.float32)).cuda()
    rec = torch.zeros((nsteps, 1, s.ny, s.nx), device="cuda")
    mms.wave_forward(s.desc, s.cf, s.m, amps, nsteps, s.fields[0], s.fields[1], rec)
    r = torch.from_numpy(g.normal(size=(nsteps, 1, s.ny, s.nx)).astype(np.float32)).cuda()
    lam = [mms.padded_empty(s.nx, s.ny, s.nz, R, nshots=1) for _ in range(2)]
    x, y, z = s.w.src[0]
    gs = s.prob.gx[x] * s.prob.gy[y] * s.prob.gz[z]
    lam_src = {}
    for n in range(nsteps, 0, -1):
        mms.wave_adjoint(s.desc, s.cf, s.m, lam[1], lam[0], r[n - 1])
        lam[0], lam[1] = lam[1], lam[0]
        lam_src[n] = lam[1][0, z + R, y + R, x + R].clone()
    ft_r = torch.stack([gs * lam_src[n + 1] if n + 1 <= nsteps else torch.zeros((), device="cuda")
                        for n in range(nsteps)]).double()
    lhs = float((rec.double() * r.double()).sum())
    rhs = float((amps[:, 0].double() * ft_r).sum())
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + abs(rhs)), (lhs, rhs)


def test_rtm512_graph_step_sampled_full_size():
    # The acoustic benchmark's configuration: 8 shots x 512^3, radius-4 FD8
    # star, 20-cell sponge, one step launched through the cached CUDA graph
    # (mms_wave_forward with MMS_WAVE_GRAPH, as the benchmark runs it),
    # teacher-forced from seeded random states and checked at sampled points
    # of every shot (source and receiver plane included) against the oracle.
    from paper_2507_11067_gb300 import _lib as L
    from paper_2507_11067_gb300.wave import WavePropagator
    n, ns = 512, 8
    w = workloads.WaveInputs(n, n, n, nshots=ns, nsteps=4, workload=4, noise=True)
    prop = WavePropagator(n, n, n, w.src, w.zrec, w.h, w.dt, sponge_width=w.sponge, sponge_a=w.sponge_a)
    prop.set_velocity(torch.from_numpy(w.v).cuda())
    m_int = oracle.model_m(w.v, w.dt, w.h)
    g = workloads.rng(4, 77)
    host = []
    for sh in range(ns):
        pair = []
        for field in (prop.p[1], prop.p[0]):      # a^n, a^{n-1}
            a = np.zeros((n + 2 * R,) * 3, np.float32)
            a[R:-R, R:-R, R:-R] = 2.0 * g.random((n, n, n), dtype=np.float32) - 1.0
            field[sh].copy_(torch.from_numpy(a))
            pair.append(a)
        host.append(pair)
    amps = torch.from_numpy(w.amp).cuda().contiguous()
    rec = torch.empty((1, ns, n, n), device="cuda")
    L.wave_forward(prop.desc, prop.coeffs, prop.m, amps[2:3], 1, prop.p[0], prop.p[1], rec, graph=True)
    torch.cuda.synchronize()
    mms.check_device()
    out = prop.p[0]                               # a^{n+1} replaced a^{n-1}
    for sh in range(ns):
        pts = workloads.sample_points(n, n, n, 600, workload=4, salt=sh)
        sx, sy, sz = w.src[sh]
        plane = np.stack([g.integers(0, n, 200), g.integers(0, n, 200), np.full(200, w.zrec)], axis=1)
        pts = np.concatenate([pts, [[sx, sy, sz]], plane]).astype(np.int64)
        ref = oracle.wave_step_points(R, workloads.fd8_star_coeffs(), m_int, (w.sponge, w.sponge_a),
                                      (sx, sy, sz), w.amp[2, sh], host[sh][0], host[sh][1], pts)
        idx = torch.from_numpy(pts).cuda()
        got = out[sh][idx[:, 2] + R, idx[:, 1] + R, idx[:, 0] + R].double().cpu().numpy()
        err = rel(got, ref)
        print(f"rtm512 graph step, shot {sh}: sampled max-rel {err:.3e}")
        assert err <= TOL, (sh, err)
        # the records are the receiver plane of the new state, bit for bit
        rp = torch.from_numpy(plane).cuda()
        assert torch.equal(rec[0, sh][rp[:, 1], rp[:, 0]], out[sh][w.zrec + R, rp[:, 1] + R, rp[:, 0] + R])


# ------------------------------------------- the gradient workload as stated
# 2 shots x 256^3, 200 steps, checkpoint every 20 (the gradient workload's own
# sizes; both checks take a few seconds at this size).

def _smooth_directions(n, count, seed, amp=30.0):
    """Seeded smooth velocity perturbations on the device: each a sum of four
    3D sinusoids with wavelengths of at least 24 cells, scaled to max |d| =
    amp m/s."""
    g = np.random.default_rng(seed)
    ax = torch.arange(n, device="cuda", dtype=torch.float32)
    z, y, x = torch.meshgrid(ax, ax, ax, indexing="ij")
    out = []
    for _ in range(count):
        d = torch.zeros((n, n, n), device="cuda")
        for _ in range(4):
            k = g.uniform(-2 * np.pi / 24, 2 * np.pi / 24, 3)
            d += float(g.uniform(0.5, 1.0)) * torch.sin(float(k[0]) * x + float(k[1]) * y + float(k[2]) * z
                                                        + float(g.uniform(0, 2 * np.pi)))
        out.append(d * (amp / d.abs().max()))
    return out


def test_gradient_fd_16_directions_full_size():
    # Central differences of J(v) = 1/2 |d(v) - d_obs|^2 along 16 seeded
    # smooth directions against the autograd gradient (hand-written adjoint,
    # checkpoint every 20 with recompute, FP64 accumulation), at rel 1e-2.
    n, ns, nsteps, every = 256, 2, 200, 20
    w_true = workloads.WaveInputs(n, n, n, nshots=ns, nsteps=nsteps, workload=5, noise=True)
    w0 = workloads.WaveInputs(n, n, n, nshots=ns, nsteps=nsteps, workload=5, noise=False)
    prop = WavePropagator(n, n, n, w0.src, w0.zrec, w0.h, w_true.dt, sponge_width=w0.sponge,
                          sponge_a=w0.sponge_a)
    amps = torch.from_numpy(w_true.amp).cuda()
    with torch.no_grad():
        obs = WaveFunction.apply(torch.from_numpy(w_true.v).cuda(), prop, amps, nsteps, every)
    v0 = torch.from_numpy(w0.v).cuda()
    v = v0.clone().requires_grad_(True)
    loss = 0.5 * ((WaveFunction.apply(v, prop, amps, nsteps, every) - obs) ** 2).sum()
    loss.backward()
    g = v.grad.double()
    torch.cuda.synchronize()
    mms.check_device()

    def records(vv):
        with torch.no_grad():
            return WaveFunction.apply(vv, prop, amps, nsteps, every).double()

    # J(v+) - J(v-) = <d+ - d-, (d+ + d-)/2 - d_obs>, exactly: summed in this
    # form the difference keeps its digits, where subtracting the two misfits
    # J(v+-) of the FP32 propagation (each far larger than their difference)
    # leaves mostly their rounding
    # The step is 0.1 of a direction (at most 3 m/s): over 200 steps the
    # records move in phase with v, and a full 30 m/s step leaves the
    # central difference about 10 % off from the nonlinearity alone.
    obs64 = obs.double()
    worst = 0.0
    for d in _smooth_directions(n, 16, seed=16):
        eps = 0.1
        dp, dm = records(v0 + eps * d), records(v0 - eps * d)
        fd = float(((dp - dm) * (0.5 * (dp + dm) - obs64)).sum()) / (2 * eps)
        an = float((g * d.double()).sum())
        worst = max(worst, abs(fd - an) / abs(an))
        assert abs(fd - an) <= 1e-2 * abs(an), (fd, an)
    print(f"gradient 2 x 256^3 x 200 steps: 16 central-difference directions, worst rel {worst:.2e}")


def _segment_dot(n, ns, K, seed):
    """<M(u, w), y> and <u, lam^1> + <w, -G^2 lam^2> for the K-step map
    M: (a^1, a^0) = (u, w) -> a^{K+1} of the wave step without sources, its
    transpose by K adjoint steps from lam^{K+1} = y, lam^{K+2} = 0 (FP64 inner
    products of the FP32 fields)."""
    w = workloads.WaveInputs(n, n, n, nshots=ns, nsteps=K, workload=5, noise=False)
    cf = workloads.fd8_star_coeffs()
    f = [mms.padded_empty(n, n, n, R, nshots=ns) for _ in range(7)]
    py, pz, ss = mms.field_geometry(f[0])
    desc, _keep = mms.wave_desc(n, n, n, R, ns, py, pz, ss, w.sponge, w.sponge_a, w.zrec, w.src)
    m = mms.padded_empty(n, n, n, R)
    mms.model_from_velocity(desc, torch.from_numpy(w.v).cuda(), m, w.dt, w.h)
    u, ww, y, cur, prev, lc, lp = f
    g = torch.Generator(device="cuda").manual_seed(seed)
    for t in (u, ww, y):
        t[:, R:-R, R:-R, R:-R] = torch.rand((ns, n, n, n), device="cuda", generator=g) * 2 - 1
    zero_amp = torch.zeros(ns, device="cuda")
    cur.copy_(u)
    prev.copy_(ww)
    for _ in range(K):
        mms.wave_step(desc, cf, m, cur, prev, zero_amp)   # prev <- a^{n+1}
        cur, prev = prev, cur
    lc.copy_(y)
    lp.zero_()
    for _ in range(K):
        mms.wave_adjoint(desc, cf, m, lc, lp)             # lp <- lam^n
        lc, lp = lp, lc
    # lc = lam^1, lp = lam^2; -G^2 lam^2 is the adjoint step with lam^{n+1} = 0
    tw = prev                                             # reuse a field buffer
    tw.copy_(lp)
    zero = mms.padded_empty(n, n, n, R, nshots=ns)
    mms.wave_adjoint(desc, cf, m, zero, tw)
    torch.cuda.synchronize()
    mms.check_device()
    lhs = _dot(_flat(cur), _flat(y))
    rhs = _dot(_flat(u), _flat(lc)) + _dot(_flat(ww), _flat(tw))
    return lhs, rhs


def test_adjoint_dot_product_one_checkpoint_segment_full_size():
    # The transpose test of the gradient workload's checkpoint segment: the
    # 20-step map of 2 shots x 256^3 against 20 adjoint steps, at rel 1e-6.
    # The 200-step map (the whole run) is printed beside it.
    lhs, rhs = _segment_dot(256, 2, 20, seed=1)
    rel20 = abs(lhs - rhs) / (abs(lhs) + abs(rhs))
    lhs2, rhs2 = _segment_dot(256, 2, 200, seed=2)
    rel200 = abs(lhs2 - rhs2) / (abs(lhs2) + abs(rhs2))
    print(f"adjoint dot test, 2 x 256^3: 20-step segment rel {rel20:.2e}, 200-step map rel {rel200:.2e}")
    assert rel20 <= 1e-6, (lhs, rhs)
    assert rel200 <= 1e-4, (lhs2, rhs2)


# --------------------------------------- the scaled adjoint (mu = m G lam)
# mms_wave_adjoint_scaled carries mu = m G lam; teacher-forced from seeded
# mu^{n+1}, mu^{n+2}, its mu^n is checked against m G lam^n of the oracle's
# adjoint step fed lam = mu / (m G), and its gradient term against the
# oracle's.

def _mg(s):
    """m G on the padded grid (FP64, zero halo) of a Setup's oracle problem."""
    p = s.prob
    g = p.gz[:, None, None] * p.gy[None, :, None] * p.gx[None, None, :]
    out = np.zeros_like(p.m)
    out[R:-R, R:-R, R:-R] = p.m[R:-R, R:-R, R:-R] * g
    return out


def _scaled_step_check(s, seed, slices=False):
    mu1, mu2, a_n, lap = s.fields
    prev, nxt = (mms.padded_empty(s.nx, s.ny, s.nz, R, nshots=s.ns) for _ in range(2))
    for f, sd in ((mu1, seed), (mu2, seed + 1), (a_n, seed + 2), (prev, seed + 3)):
        s.fill(f, sd)
    mms.wave_step_lap(s.desc, s.cf, s.m, a_n, prev, nxt, lap, s.amps[0])      # L a^n
    m1, m2, an = s.host(mu1), s.host(mu2), s.host(a_n)
    g = np.random.default_rng(seed + 4)
    resid = torch.from_numpy(g.normal(size=(s.ns, s.ny, s.nx)).astype(np.float32)).cuda()
    n3 = (s.nz, s.ny, s.nx)
    if slices:   # every shot its own FP64 slice, summed afterwards
        py, pz, ss = mms.field_geometry(s.fields[0])
        desc, _keep = mms.wave_desc(s.nx, s.ny, s.nz, R, s.ns, py, pz, ss, s.w.sponge, s.w.sponge_a, s.w.zrec,
                                    s.w.src, grad_shot_stride=s.nx * s.ny * s.nz)
        gs = torch.zeros((s.ns,) + n3, device="cuda", dtype=torch.float64)
        mms.wave_adjoint_scaled(desc, s.cf, s.m, mu1, mu2, resid, lap, gs)
        grad = torch.zeros(n3, device="cuda", dtype=torch.float64)
        mms.sum_f64(gs, grad)
    else:
        grad = torch.zeros(n3, device="cuda", dtype=torch.float64)
        mms.wave_adjoint_scaled(s.desc, s.cf, s.m, mu1, mu2, resid, lap, grad)
    mms.grad_divide_m(s.desc, s.m, grad)        # the sum of mu^{n+1} (L a^n) over m
    torch.cuda.synchronize()
    mms.check_device()
    got = mu2.cpu().numpy()
    mg = _mg(s)
    inner = mg > 0
    rh = resid.cpu().numpy().astype(np.float64)
    gref = np.zeros((s.nz, s.ny, s.nx))
    errs = []
    for sh in range(s.ns):
        l1 = np.divide(m1[sh], mg, out=np.zeros_like(mg), where=inner)
        l2 = np.divide(m2[sh], mg, out=np.zeros_like(mg), where=inner)
        ref = mg * s.prob.adjoint_step(l1, l2, rh[sh], an[sh], gref)
        errs.append(rel(got[sh], ref))
    return errs, rel(grad.cpu().numpy(), gref)


@pytest.mark.parametrize("nshots,slices", [(1, False), (2, False), (3, False), (4, False), (2, True), (3, True)])
def test_scaled_adjoint_step_against_oracle(nshots, slices):
    # one shot per CTA; the shots' gradient terms meet in one shared FP64
    # slice (atomics) or in per-shot slices summed afterwards
    s = Setup(nshots=nshots)
    errs, eg = _scaled_step_check(s, 70, slices=slices)
    print(f"scaled adjoint step, {nshots} shots{' (slices)' if slices else ''}: mu^n max-rel {max(errs):.2e}, "
          f"gradient term {eg:.2e}")
    assert max(errs) <= TOL and eg <= TOL


@pytest.mark.parametrize("nshots", [1, 3])
def test_scaled_adjoint_step_bulk_rows(nshots):
    # an even nx: the shared slice's rows are added by bulk reductions (the
    # odd nx above takes one atomic per point); nx = 70 leaves a last tile
    # of 6 points, and three shots reduce into the same rows
    s = Setup(nx=70, ny=38, nz=41, nshots=nshots)
    errs, eg = _scaled_step_check(s, 75)
    print(f"scaled adjoint step, nx 70, {nshots} shots: mu^n max-rel {max(errs):.2e}, gradient term {eg:.2e}")
    assert max(errs) <= TOL and eg <= TOL


def test_scaled_adjoint_step_full_size():
    # the gradient workload's size (2 shots x 256^3, 20-cell sponge), every point
    s = Setup(nx=256, ny=256, nz=256, nshots=2, nsteps=4, sponge=20, seed=3)
    errs, eg = _scaled_step_check(s, 80)
    print(f"scaled adjoint step 256^3: mu^n max-rel {max(errs):.2e}, gradient term {eg:.2e}")
    assert max(errs) <= TOL and eg <= TOL


@pytest.mark.parametrize("form", ["lam", "mu"])
def test_gradient_term_widening_is_exact_for_subnormal_products(form):
    # One shot, no sponge (G = 1): the gradient term of one adjoint step is
    # the FP32 product lam^{n+1} (L a^n) (or mu^{n+1} (L a^n)) widened to
    # FP64 and added to zero, so it must equal, bit for bit, numpy's IEEE
    # FP32 arithmetic converted with a true (double) -- here on operands
    # whose products fall among the FP32 denormals (below 1.2e-38) as well as
    # normal ones.
    nx, ny, nz = 40, 36, 24
    w = workloads.WaveInputs(nx, ny, nz, nshots=1, nsteps=2, workload=5, sponge=0, salt=9)
    m = mms.padded_empty(nx, ny, nz, R)
    f = [mms.padded_empty(nx, ny, nz, R, nshots=1) for _ in range(3)]
    py, pz, ss = mms.field_geometry(f[0])
    desc, _keep = mms.wave_desc(nx, ny, nz, R, 1, py, pz, ss, 0, 0.0, -1, w.src)
    mms.model_from_velocity(desc, torch.from_numpy(w.v).cuda(), m, w.dt, w.h)
    g = np.random.default_rng(12)
    n3 = (nz, ny, nx)
    sign = lambda: np.where(g.random(n3) < 0.5, -1.0, 1.0)  # noqa: E731
    # magnitudes 1e-24 .. 1e-14 for the state and 1e-24 .. 1e-19 for L a^n:
    # products from 1e-48 (rounds to zero) through the denormals to 1e-33
    x1 = (sign() * 10.0 ** g.uniform(-24, -14, n3)).astype(np.float32)
    xl = (sign() * 10.0 ** g.uniform(-24, -19, n3)).astype(np.float32)
    cur, prev, lap = f
    cur[0, R:-R, R:-R, R:-R] = torch.from_numpy(x1)
    lap[0, R:-R, R:-R, R:-R] = torch.from_numpy(xl)
    grad = torch.zeros(n3, device="cuda", dtype=torch.float64)
    fn = mms.wave_adjoint_lap if form == "lam" else mms.wave_adjoint_scaled
    fn(desc, workloads.fd8_star_coeffs(), m, cur, prev, None, lap, grad)
    term = x1 * xl
    torch.cuda.synchronize()
    mms.check_device()
    assert term.dtype == np.float32
    tiny = np.finfo(np.float32).tiny
    denormal = (term != 0) & (np.abs(term) < tiny)
    assert denormal.sum() > 1000 and (np.abs(term) >= tiny).sum() > 1000
    got = grad.cpu().numpy()
    exact = term.astype(np.float64)
    assert np.array_equal(got, exact), float(np.abs(got - exact).max())


def test_gradient_scaled_and_lambda_forms_agree():
    # the two adjoint variables give the same gradient of the 48^3 workload
    w_true, w0 = _grad_problem()
    n, nsteps, every = 48, 200, 20
    prop = WavePropagator(n, n, n, w0.src, w0.zrec, w0.h, w_true.dt, sponge_width=w0.sponge,
                          sponge_a=w0.sponge_a)
    amps = torch.from_numpy(w_true.amp).cuda()
    with torch.no_grad():
        obs, _ = prop.forward(torch.from_numpy(w_true.v).cuda(), amps, nsteps)
        rec, ckpt = prop.forward(torch.from_numpy(w0.v).cuda(), amps, nsteps, ckpt_every=every)
    out = [prop.gradient_m(amps, rec - obs, ckpt, every, scaled=sc).cpu().numpy() for sc in (True, False)]
    torch.cuda.synchronize()
    mms.check_device()
    err = rel(out[0], out[1])
    print(f"gradient 48^3: mu form vs lam form max-rel {err:.2e}")
    assert err <= 1e-4
