"""GPU parity of the VTI and TTI steps against the FP64 oracle (oracle/aniso.py).

Teacher-forced: the oracle takes the GPU's FP32 states and medium inputs
and does one FP64 step; the bar is max|gpu - oracle| / max|oracle| <= 1e-5
for one step (FP32 arithmetic over at most 2 x 17 terms per point).
"""
import numpy as np
import pytest

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
    return float(np.abs(np.asarray(g, np.float64) - o).max() / max(np.abs(o).max(), 1e-300))


class Vti:
    def __init__(self, nx=45, ny=38, nz=41, r=4, nshots=2, sponge=6, seed=0, nsteps=30, rec=True):
        self.nx, self.ny, self.nz, self.r, self.ns = nx, ny, nz, r, nshots
        self.a = workloads.AnisoInputs(nx, ny, nz, nshots, nsteps, sponge=sponge, salt=seed)
        g = np.random.default_rng(100 + seed)
        # per-point medium (the workload's eps, delta are per layer): every
        # coefficient varies from point to point here
        self.eps = g.uniform(0.0, 0.3, (nz, ny, nx)).astype(np.float32)
        self.delta = g.uniform(-0.1, 0.2, (nz, ny, nx)).astype(np.float32)
        self.vp = self.a.vp
        self.cf = workloads.fd8_star_coeffs() if r == 4 else workloads.normal_coeffs("star", r, workload=6,
                                                                                     salt=seed)
        self.mv = mms.padded_empty(nx, ny, nz, r)
        self.rho = mms.padded_empty(nx, ny, nz, r)
        self.f = [mms.padded_empty(nx, ny, nz, r, nshots=nshots) for _ in range(6)]
        py, pz, ss = mms.field_geometry(self.f[0])
        self.desc, self._src = mms.wave_desc(nx, ny, nz, r, nshots, py, pz, ss, sponge, self.a.wave.sponge_a,
                                             self.a.zrec if rec else -1, self.a.src)
        dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
        mms.vti_model(self.desc, dev(self.vp), dev(self.eps), dev(self.delta), self.mv, self.rho, self.a.dt,
                      self.a.h)
        self.amps = torch.from_numpy(self.a.amp).cuda().contiguous()
        self.mh_o, self.mv_o = aniso.vti_medium(self.vp, self.eps, self.delta, self.a.dt, self.a.h)
        self.sponge = (sponge, self.a.wave.sponge_a) if sponge else None

    def fill(self, f, seed):
        g = np.random.default_rng(seed)
        r = self.r
        f[:, r:-r, r:-r, r:-r] = torch.from_numpy(
            g.uniform(-1, 1, (self.ns, self.nz, self.ny, self.nx)).astype(np.float32))

    def oracle_step(self, hc, vc, hp, vp, n, sh):
        return aniso.vti_step(self.r, self.cf, self.mh_o, self.mv_o, self.sponge, self.a.src[sh],
                              float(self.a.amp[n, sh]), hc[sh], vc[sh], hp[sh], vp[sh])


def _host(t):
    return t.cpu().numpy().astype(np.float64)


def test_vti_model_matches_the_oracle_medium():
    s = Vti()
    r = s.r
    mv = s.mv.cpu().numpy()
    rho = s.rho.cpu().numpy()
    assert rel(mv[r:-r, r:-r, r:-r], s.mv_o) <= 1e-6
    assert rel(rho[r:-r, r:-r, r:-r], s.mh_o / s.mv_o) <= 1e-6
    assert np.all(mv[:r] == 0) and np.all(rho[:, :, :r] == 0)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_vti_teacher_forced_step(r):
    s = Vti(nx=45 + r, ny=38, nz=41 - r, r=r, seed=r)
    hc, vc, hp, vp, hn, vn = s.f
    for k, f in enumerate((hc, vc, hp, vp)):
        s.fill(f, 10 * r + k)
    # a source value that stands out, so that a misplaced source fails
    s.amps[7] = 3.0
    s.a.amp[7] = 3.0
    rec = torch.zeros((s.ns, s.ny, s.nx), device="cuda")
    ins = [_host(f) for f in (hc, vc, hp, vp)]
    mms.vti_step(s.desc, s.cf, s.mv, s.rho, hc, vc, hp, vp, hn, vn, s.amps[7], rec)
    torch.cuda.synchronize()
    mms.check_device()
    gh, gv = _host(hn), _host(vn)
    for sh in range(s.ns):
        oh, ov = s.oracle_step(*ins, 7, sh)
        eh, ev = rel(gh[sh], oh), rel(gv[sh], ov)
        print(f"VTI r={r} shot {sh}: sigma_H {eh:.2e}, sigma_V {ev:.2e}")
        assert eh <= TOL and ev <= TOL
        # halos untouched (zero), records = sigma_H on the receiver plane
        assert np.all(gh[sh][:r] == 0) and np.all(gv[sh][:, :, -r:] == 0)
        np.testing.assert_array_equal(rec[sh].cpu().numpy(), hn[sh, r + s.a.zrec, r:-r, r:-r].cpu().numpy())


def test_vti_in_place_equals_out_of_place_and_every_variant_agrees():
    s = Vti(nx=70, ny=37, nz=45, nshots=1, rec=False)
    hc, vc, hp, vp, hn, vn = s.f
    for k, f in enumerate((hc, vc, hp, vp)):
        s.fill(f, 40 + k)
    ins = [_host(f) for f in (hc, vc, hp, vp)]
    oh, ov = s.oracle_step(*ins, 5, 0)
    nvar = mms.aniso_num_variants("vti")
    assert nvar >= 2
    try:
        for v in range(nvar):
            mms.aniso_set_variant("vti", v)
            mms.vti_step(s.desc, s.cf, s.mv, s.rho, hc, vc, hp, vp, hn, vn, s.amps[5])
            hp2 = mms.padded_empty(s.nx, s.ny, s.nz, s.r, nshots=1)
            vp2 = mms.padded_empty(s.nx, s.ny, s.nz, s.r, nshots=1)
            hp2.copy_(hp)
            vp2.copy_(vp)
            mms.vti_step(s.desc, s.cf, s.mv, s.rho, hc, vc, hp2, vp2, hp2, vp2, s.amps[5])
            torch.cuda.synchronize()
            mms.check_device()
            assert torch.equal(hp2, hn) and torch.equal(vp2, vn), v
            eh, ev = rel(_host(hn)[0], oh), rel(_host(vn)[0], ov)
            print(f"VTI variant {v}: {eh:.2e} {ev:.2e}")
            assert eh <= TOL and ev <= TOL, v
    finally:
        mms.aniso_set_variant("vti", 0)
    with pytest.raises(mms.MMSError):
        mms.aniso_set_variant("vti", nvar)


def test_vti_trajectory_from_rest():
    # 40 steps from zero states with the Ricker source; the oracle runs the
    # same steps in FP64 from its own states (not teacher-forced)
    s = Vti(nx=48, ny=44, nz=40, nshots=2, sponge=8, nsteps=40)
    hc, vc, hp, vp, hn, vn = s.f
    r = s.r
    oh = [[np.zeros(hc.shape[1:]) for _ in range(4)] for _ in range(s.ns)]   # hc, vc, hp, vp per shot
    cur = [hc, vc, hp, vp]
    for n in range(40):
        mms.vti_step(s.desc, s.cf, s.mv, s.rho, cur[0], cur[1], cur[2], cur[3], cur[2], cur[3], s.amps[n])
        cur = [cur[2], cur[3], cur[0], cur[1]]
        for sh in range(s.ns):
            h1, v1 = aniso.vti_step(r, s.cf, s.mh_o, s.mv_o, s.sponge, s.a.src[sh], float(s.a.amp[n, sh]),
                                    *oh[sh])
            oh[sh] = [h1, v1, oh[sh][0], oh[sh][1]]
    torch.cuda.synchronize()
    mms.check_device()
    gh, gv = _host(cur[0]), _host(cur[1])
    for sh in range(s.ns):
        eh, ev = rel(gh[sh], oh[sh][0]), rel(gv[sh], oh[sh][1])
        print(f"VTI 40-step trajectory shot {sh}: {eh:.2e} {ev:.2e}")
        assert np.abs(oh[sh][0]).max() > 0
        assert eh <= 1e-4 and ev <= 1e-4


def test_vti_refuses_overlaps_and_bad_alignment():
    s = Vti(nx=20, ny=20, nz=20, nshots=1)
    hc, vc, hp, vp, hn, vn = s.f
    with pytest.raises(mms.MMSError):
        mms.vti_step(s.desc, s.cf, s.mv, s.rho, hc, hc, hp, vp, hn, vn, s.amps[0])
    with pytest.raises(mms.MMSError):
        mms.vti_step(s.desc, s.cf, s.mv, s.rho, hc, vc, hp, vp, hn, hn, s.amps[0])
    with pytest.raises(mms.MMSError):
        mms.vti_step(s.desc, s.cf, s.mv, s.rho, hc, vc, hp, vp, vp, vn, s.amps[0])   # next over the other prev
    # a field one float off the 16-byte grid, with room for its whole geometry
    flat = torch.zeros(hc.untyped_storage().nbytes() // 4 + 4, device="cuda")
    mis = torch.as_strided(flat, hc.shape, hc.stride(), 1)
    with pytest.raises(mms.MMSError, match="E_ALIGN"):
        mms.vti_step(s.desc, s.cf, s.mv, s.rho, mis, vc, hp, vp, hn, vn, s.amps[0])


def test_vti_512_sampled_full_size():
    # the bench's grid (512^3, r = 4, FD8, one shot here), checked at sampled
    # points against the oracle's point-wise step
    n = 512
    a = workloads.AnisoInputs(n, n, n, 1, 4, workload=6)
    r = 4
    cf = workloads.fd8_star_coeffs()
    mv, rho = mms.padded_empty(n, n, n, r), mms.padded_empty(n, n, n, r)
    f = [mms.padded_empty(n, n, n, r, nshots=1) for _ in range(4)]
    py, pz, ss = mms.field_geometry(f[0])
    desc, _src = mms.wave_desc(n, n, n, r, 1, py, pz, ss, 20, a.wave.sponge_a, a.zrec, a.src)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    mms.vti_model(desc, dev(a.vp), dev(a.eps), dev(a.delta), mv, rho, a.dt, a.h)
    g = np.random.default_rng(9)
    host = []
    for k in range(4):
        x = np.zeros(f[k].shape[1:], np.float32)
        x[r:-r, r:-r, r:-r] = g.uniform(-1, 1, (n, n, n)).astype(np.float32)
        f[k][0].copy_(torch.from_numpy(x))
        host.append(x)
    amp = torch.full((1,), 2.5, device="cuda")
    hn = mms.padded_empty(n, n, n, r, nshots=1, zero=False)
    vn = mms.padded_empty(n, n, n, r, nshots=1, zero=False)
    mms.vti_step(desc, cf, mv, rho, f[0], f[1], f[2], f[3], hn, vn, amp)
    torch.cuda.synchronize()
    mms.check_device()
    pts = np.vstack([workloads.sample_points(n, n, n, 3000, workload=6), [a.src[0]]])
    mh_o, mv_o = aniso.vti_medium(a.vp, a.eps, a.delta, a.dt, a.h)
    oh, ov = aniso.vti_step_points(r, cf, mh_o, mv_o, (20, a.wave.sponge_a), a.src[0], 2.5, *host, pts)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    gh = hn[0].cpu().numpy()[z + r, y + r, x + r]
    gv = vn[0].cpu().numpy()[z + r, y + r, x + r]
    eh, ev = rel(gh, oh), rel(gv, ov)
    print(f"VTI 512^3 sampled ({len(pts)} points): {eh:.2e} {ev:.2e}")
    assert eh <= TOL and ev <= TOL


# ------------------------------------------------------------------ TTI

class Tti:
    def __init__(self, nx=45, ny=38, nz=41, r=4, nshots=2, sponge=6, seed=0, nsteps=30, rec=True):
        self.nx, self.ny, self.nz, self.r, self.ns = nx, ny, nz, r, nshots
        self.a = workloads.AnisoInputs(nx, ny, nz, nshots, nsteps, workload=7, sponge=sponge, salt=seed, tti=True)
        g = np.random.default_rng(200 + seed)
        n3 = (nz, ny, nx)
        # per-point medium and tilt: every coefficient of H1 and of the
        # coupling varies from point to point
        self.inputs = [self.a.vp, (0.4 * self.a.vp * g.uniform(0.9, 1.1, n3)).astype(np.float32),
                       g.uniform(0.0, 0.3, n3).astype(np.float32), g.uniform(-0.1, 0.2, n3).astype(np.float32),
                       g.uniform(0.7, 1.3, n3).astype(np.float32), g.uniform(0.0, np.pi / 2, n3).astype(np.float32),
                       g.uniform(-np.pi, np.pi, n3).astype(np.float32)]
        self.w2 = aniso.fd2_row(r).astype(np.float32)
        self.w1 = aniso.fd1_row(r).astype(np.float32)
        self.med = torch.empty((8, nz, ny, nx), device="cuda")
        self.work = torch.empty((4, nshots, nz, ny, nx), device="cuda")
        self.f = [mms.padded_empty(nx, ny, nz, r, nshots=nshots) for _ in range(6)]
        py, pz, ss = mms.field_geometry(self.f[0])
        self.desc, self._src = mms.wave_desc(nx, ny, nz, r, nshots, py, pz, ss, sponge, self.a.wave.sponge_a,
                                             self.a.zrec if rec else -1, self.a.src)
        dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in self.inputs]
        mms.tti_model(self.desc, *dev, self.med, self.a.dt, self.a.h)
        self.amps = torch.from_numpy(self.a.amp).cuda().contiguous()
        vp, vs, eps, delta, alpha, th, ph = self.inputs
        self.med_o = aniso.tti_medium(vp, vs, eps, delta, alpha, self.a.dt, self.a.h)
        self.tilt_o = aniso.tilt_axis(th, ph)
        self.sponge = (sponge, self.a.wave.sponge_a) if sponge else None

    fill = Vti.fill

    def step(self, pc, qc, pp, qp, pn, qn, amp, rec=None):
        mms.tti_step(self.desc, self.w2, self.w1, self.med, pc, qc, pp, qp, pn, qn, self.work, amp, rec)

    def oracle_step(self, pc, qc, pp, qp, n, sh):
        return aniso.tti_step(self.r, self.med_o, self.tilt_o, self.sponge, self.a.src[sh], float(self.a.amp[n, sh]),
                              pc[sh], qc[sh], pp[sh], qp[sh], self.w2, self.w1)


def test_tti_model_matches_the_oracle_medium():
    s = Tti()
    med = s.med.cpu().numpy().astype(np.float64)
    for k in range(5):
        assert rel(med[k], s.med_o[k]) <= 1e-6, k
    for k in range(3):
        assert np.abs(med[5 + k] - s.tilt_o[k]).max() <= 1e-6, k


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_tti_teacher_forced_step(r):
    s = Tti(nx=45 + r, ny=38, nz=41 - r, r=r, seed=r)
    pc, qc, pp, qp, pn, qn = s.f
    for k, f in enumerate((pc, qc, pp, qp)):
        s.fill(f, 30 * r + k)
    s.amps[4] = 3.0
    s.a.amp[4] = 3.0
    rec = torch.zeros((s.ns, s.ny, s.nx), device="cuda")
    ins = [_host(f) for f in (pc, qc, pp, qp)]
    s.step(pc, qc, pp, qp, pn, qn, s.amps[4], rec)
    torch.cuda.synchronize()
    mms.check_device()
    gp, gq = _host(pn), _host(qn)
    for sh in range(s.ns):
        op, oq = s.oracle_step(*ins, 4, sh)
        ep, eq = rel(gp[sh], op), rel(gq[sh], oq)
        print(f"TTI r={r} shot {sh}: p {ep:.2e}, q {eq:.2e}")
        assert ep <= TOL and eq <= TOL
        assert np.all(gp[sh][:r] == 0) and np.all(gq[sh][:, :, -r:] == 0)
        np.testing.assert_array_equal(rec[sh].cpu().numpy(), pn[sh, r + s.a.zrec, r:-r, r:-r].cpu().numpy())


@pytest.mark.parametrize("nx", [70, 72])   # separate combine (nx % 4 != 0) and the fused q pass
def test_tti_in_place_equals_out_of_place(nx):
    s = Tti(nx=nx, ny=37, nz=45, nshots=1, rec=False)
    pc, qc, pp, qp, pn, qn = s.f
    for k, f in enumerate((pc, qc, pp, qp)):
        s.fill(f, 60 + k)
    s.step(pc, qc, pp, qp, pn, qn, s.amps[3])
    pp2 = mms.padded_empty(s.nx, s.ny, s.nz, s.r, nshots=1)
    qp2 = mms.padded_empty(s.nx, s.ny, s.nz, s.r, nshots=1)
    pp2.copy_(pp)
    qp2.copy_(qp)
    s.step(pc, qc, pp2, qp2, pp2, qp2, s.amps[3])
    torch.cuda.synchronize()
    mms.check_device()
    assert torch.equal(pp2, pn) and torch.equal(qp2, qn)
    ins = [_host(f) for f in (pc, qc, pp, qp)]
    op, oq = s.oracle_step(*ins, 3, 0)
    ep, eq = rel(_host(pn)[0], op), rel(_host(qn)[0], oq)
    print(f"TTI nx={nx}: {ep:.2e} {eq:.2e}")
    assert ep <= TOL and eq <= TOL


def test_tti_trajectory_from_rest():
    s = Tti(nx=48, ny=44, nz=40, nshots=2, sponge=8, nsteps=30)
    pc, qc, pp, qp, pn, qn = s.f
    r = s.r
    o = [[np.zeros(pc.shape[1:]) for _ in range(4)] for _ in range(s.ns)]
    cur = [pc, qc, pp, qp]
    for n in range(30):
        s.step(cur[0], cur[1], cur[2], cur[3], cur[2], cur[3], s.amps[n])
        cur = [cur[2], cur[3], cur[0], cur[1]]
        for sh in range(s.ns):
            p1, q1 = aniso.tti_step(r, s.med_o, s.tilt_o, s.sponge, s.a.src[sh], float(s.a.amp[n, sh]), *o[sh],
                                    s.w2, s.w1)
            o[sh] = [p1, q1, o[sh][0], o[sh][1]]
    torch.cuda.synchronize()
    mms.check_device()
    gp, gq = _host(cur[0]), _host(cur[1])
    for sh in range(s.ns):
        ep, eq = rel(gp[sh], o[sh][0]), rel(gq[sh], o[sh][1])
        print(f"TTI 30-step trajectory shot {sh}: {ep:.2e} {eq:.2e}")
        assert np.abs(o[sh][0]).max() > 0
        assert ep <= 1e-4 and eq <= 1e-4


def test_tti_refuses_bad_work_and_weights():
    s = Tti(nx=20, ny=20, nz=20, nshots=1)
    pc, qc, pp, qp, pn, qn = s.f
    with pytest.raises(mms.MMSError):       # work over an output field
        mms.tti_step(s.desc, s.w2, s.w1, s.med, pc, qc, pp, qp, pn, qn, pn, s.amps[0])
    with pytest.raises(mms.MMSError):       # outputs overlap
        mms.tti_step(s.desc, s.w2, s.w1, s.med, pc, qc, pp, qp, pn, pn, s.work, s.amps[0])
    with pytest.raises(ValueError):
        mms.tti_step(s.desc, s.w2[:-1], s.w1, s.med, pc, qc, pp, qp, pn, qn, s.work, s.amps[0])


def test_tti_512_sampled_full_size():
    n, r = 512, 4
    a = workloads.AnisoInputs(n, n, n, 1, 4, workload=7, tti=True)
    w2 = aniso.fd2_row(r).astype(np.float32)
    w1 = aniso.fd1_row(r).astype(np.float32)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    med = torch.empty((8, n, n, n), device="cuda")
    f = [mms.padded_empty(n, n, n, r, nshots=1) for _ in range(4)]
    py, pz, ss = mms.field_geometry(f[0])
    desc, _src = mms.wave_desc(n, n, n, r, 1, py, pz, ss, 20, a.wave.sponge_a, a.zrec, a.src)
    mms.tti_model(desc, dev(a.vp), dev(a.vs), dev(a.eps), dev(a.delta), dev(a.alpha), dev(a.theta), dev(a.phi),
                  med, a.dt, a.h)
    g = np.random.default_rng(19)
    host = []
    for k in range(4):
        x = np.zeros(f[k].shape[1:], np.float32)
        x[r:-r, r:-r, r:-r] = g.uniform(-1, 1, (n, n, n)).astype(np.float32)
        f[k][0].copy_(torch.from_numpy(x))
        host.append(x)
    work = torch.empty((4, 1, n, n, n), device="cuda")
    pn = mms.padded_empty(n, n, n, r, nshots=1, zero=False)
    qn = mms.padded_empty(n, n, n, r, nshots=1, zero=False)
    amp = torch.full((1,), 2.5, device="cuda")
    mms.tti_step(desc, w2, w1, med, f[0], f[1], f[2], f[3], pn, qn, work, amp)
    torch.cuda.synchronize()
    mms.check_device()
    pts = np.vstack([workloads.sample_points(n, n, n, 2000, workload=7), [a.src[0]]])
    med_o = aniso.tti_medium(a.vp, a.vs, a.eps, a.delta, a.alpha, a.dt, a.h)
    tilt_o = aniso.tilt_axis(a.theta, a.phi)
    op, oq = aniso.tti_step_points(r, med_o, tilt_o, (20, a.wave.sponge_a), a.src[0], 2.5, *host, pts, w2, w1)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    gp = pn[0].cpu().numpy()[z + r, y + r, x + r]
    gq = qn[0].cpu().numpy()[z + r, y + r, x + r]
    ep, eq = rel(gp, op), rel(gq, oq)
    print(f"TTI 512^3 sampled ({len(pts)} points): {ep:.2e} {eq:.2e}")
    assert ep <= TOL and eq <= TOL
