"""Pins of the FP64 wave-step oracle and its adjoint.

The step is checked against conservation laws and special cases that fix it
independently of oracle.c (energy, time reversal, a scalar recurrence, the
sponge's closed form); the adjoint against the forward (dot-product tests)
and the gradient against finite differences of the forward objective.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

R = 4


def _problem(n=(10, 9, 11), sponge=None, seed=0, nsteps=40, vjit=0.0, src=None):
    nz, ny, nx = n
    g = np.random.default_rng(seed)
    v = 2000.0 * (1.0 + vjit * g.uniform(-1, 1, size=n))
    h, dt = 10.0, 0.4 * 10.0 / float(np.max(v))
    m = oracle.model_m(v, dt, h)
    src = src or [(nx // 2, ny // 2, nz // 2)]
    amp = np.zeros((nsteps, len(src)))
    t = np.arange(nsteps) * dt
    amp[:, :] = (dt * dt * workloads.ricker(t, 60.0, 1.0 / 60.0))[:, None]
    return oracle.WaveProblem(R, oracle.fd2_star_coeffs(R), m, sponge, src, amp, zrec=1), v, dt, h


def test_sponge_closed_form():
    g = oracle.sponge_1d(50, 20, 0.015)
    assert g[0] == pytest.approx(math.exp(-(0.015 * 20) ** 2), rel=1e-15)
    assert g[19] == pytest.approx(math.exp(-(0.015 * 1) ** 2), rel=1e-15)
    assert g[49] == g[0] and g[30] == g[19]
    assert np.all(g[20:30] == 1.0)
    assert np.all(np.diff(g[:21]) > 0)


def test_step_scalar_recurrence_without_stencil():
    # With all weights zero, L = 0 and each point follows
    # a^{n+1} = g (2 a^n - g a^{n-1} + s^n): check the source point.
    p, *_ = _problem(sponge=(3, 0.2), nsteps=12)
    p.c[:] = 0.0
    a_prev, a_cur = p.zeros(), p.zeros()
    sx, sy, sz = p.src[0]
    gsrc = p.gx[sx] * p.gy[sy] * p.gz[sz]
    x1, x0 = 0.0, 0.0
    for n in range(12):
        a_next = p.step(a_cur, a_prev, 0, n)
        x1, x0 = gsrc * (2 * x1 - gsrc * x0 + p.amp[n, 0]), x1
        assert a_next[sz + R, sy + R, sx + R] == pytest.approx(x1, rel=1e-14, abs=1e-300)
        a_prev, a_cur = a_cur, a_next
    assert np.count_nonzero(a_cur) == 1


def _energy(p, a1, a0):
    d = (a1 - a0)[R:-R, R:-R, R:-R]
    mi = p.m[R:-R, R:-R, R:-R]
    return np.sum(d * d / mi) - np.sum(a1[R:-R, R:-R, R:-R] * p.laplacian(a0))


def test_energy_conserved_without_sponge():
    # G = 1, source off after it has fired: E^{n+1/2} =
    # <a^{n+1}-a^n, m^{-1}(a^{n+1}-a^n)> - <a^{n+1}, L a^n> is invariant.
    p, *_ = _problem(nsteps=300, vjit=0.3, seed=1)
    p.amp[40:] = 0.0
    a0, a1 = p.zeros(), p.zeros()
    E = []
    for n in range(300):
        a0, a1 = a1, p.step(a1, a0, 0, n)
        if n >= 41:
            E.append(_energy(p, a1, a0))
    E = np.array(E)
    assert E[0] > 0
    assert np.abs(E - E[0]).max() <= 1e-10 * E[0]


def test_energy_decays_with_sponge():
    p, *_ = _problem(nsteps=200, sponge=(3, 0.3), seed=2)
    p.amp[40:] = 0.0
    a0, a1 = p.zeros(), p.zeros()
    E = []
    for n in range(200):
        a0, a1 = a1, p.step(a1, a0, 0, n)
        if n >= 41:
            E.append(_energy(p, a1, a0))
    assert E[-1] < 0.5 * E[0]


def test_time_reversibility():
    # Without sponge and source: a^{n-1} = (2 + m L) a^n - a^{n+1}.
    p, *_ = _problem(nsteps=60, seed=3, vjit=0.2)
    a0, a1 = p.zeros(), p.zeros()
    hist = [a0, a1]
    for n in range(60):
        a0, a1 = a1, p.step(a1, a0, 0, n)
        hist.append(a1)
    p.amp[:] = 0.0
    # walk back 30 steps from the last two states using the forward step with
    # the roles of past and future exchanged
    cur, nxt = hist[-2], hist[-1]
    for k in range(30):
        prev = p.step(cur, nxt, 0, 0)   # (2 + mL) cur - nxt
        ref = hist[-3 - k]
        assert np.abs(prev - ref).max() <= 1e-9 * np.abs(ref).max()
        nxt, cur = cur, prev


@pytest.mark.parametrize("ratio,grows", [(0.97, False), (1.03, True)])
def test_cfl_bound(ratio, grows):
    # Leapfrog with the FD8 star is stable iff v dt / h <= 2/sqrt(3*2048/315).
    bound = 2.0 / math.sqrt(3 * 2048 / 315)
    n = (12, 12, 12)
    m = np.full(n, (ratio * bound) ** 2)
    amp = np.zeros((400, 1))
    p = oracle.WaveProblem(R, oracle.fd2_star_coeffs(R), m, None, [(6, 6, 6)], amp, zrec=0)
    g = np.random.default_rng(0)
    a0 = oracle.pad(g.uniform(-1, 1, size=n), R)
    a1 = a0.copy()
    for k in range(400):
        a0, a1 = a1, p.step(a1, a0, 0, k)
    peak = np.abs(a1).max()
    assert (peak > 1e3) == grows


def test_records_are_receiver_plane():
    p, *_ = _problem(nsteps=15, sponge=(2, 0.2), src=[(3, 4, 2), (7, 5, 6)])
    rec, states = p.forward(15, keep_states=True)
    for s in range(2):
        for n in (1, 8, 15):
            assert np.array_equal(rec[n - 1, s], states[s][n][R + p.zrec, R:-R, R:-R])
    assert np.abs(rec[:, 0] - rec[:, 1]).max() > 0


def test_adjoint_one_step_dot_product():
    # One step T(u, w) = G(2 + M L) u - G^2 w, with adjoint
    # T^T lam = ((2 + L M) G lam, -G^2 lam), from adjoint_step.
    p, *_ = _problem(sponge=(3, 0.3), vjit=0.3, seed=4)
    p.amp[:] = 0.0
    g = np.random.default_rng(6)
    u = oracle.pad(g.normal(size=(p.nz, p.ny, p.nx)), R)
    w = oracle.pad(g.normal(size=(p.nz, p.ny, p.nx)), R)
    lam = oracle.pad(g.normal(size=(p.nz, p.ny, p.nx)), R)
    Tuw = p.step(u, w, 0, 0)
    dummy = np.zeros((p.nz, p.ny, p.nx))
    tu = p.adjoint_step(lam, p.zeros(), None, None, dummy)
    tw = p.adjoint_step(p.zeros(), lam, None, None, dummy)
    lhs = p.dot(Tuw, lam)
    rhs = p.dot(u, tu) + p.dot(w, tw)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(p.dot(u, tu)) + abs(p.dot(w, tw)))


def test_adjoint_full_map_dot_product():
    # Source series s -> records d is linear, d = F s.  Its adjoint from the
    # adjoint recursion: (F^T r)^n = g_src * lam^{n+1}[src].
    nsteps = 50
    p, *_ = _problem(sponge=(3, 0.3), vjit=0.3, seed=5, nsteps=nsteps)
    g = np.random.default_rng(8)
    s = g.normal(size=nsteps)
    p.amp[:, 0] = s
    rec, _ = p.forward(nsteps)
    rres = g.normal(size=rec.shape)
    lam1, lam2 = p.zeros(), p.zeros()
    lams = {}
    dummy = np.zeros((p.nz, p.ny, p.nx))
    for n in range(nsteps, 0, -1):
        lam0 = p.adjoint_step(lam1, lam2, rres[n - 1, 0], None, dummy)
        lams[n] = lam0
        lam2, lam1 = lam1, lam0
    sx, sy, sz = p.src[0]
    gs = p.gx[sx] * p.gy[sy] * p.gz[sz]
    Ft_r = np.array([gs * lams[n + 1][sz + R, sy + R, sx + R] for n in range(nsteps)])
    lhs = np.sum(rec * rres)
    rhs = np.sum(s * Ft_r)
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(rec * rres))


def _objective_at(m_int, base, obs, nsteps):
    p = oracle.WaveProblem(R, base.c.reshape(3, -1), m_int, None, base.src, base.amp, base.zrec)
    p.gx, p.gy, p.gz = base.gx, base.gy, base.gz
    rec, _ = p.forward(nsteps)
    return oracle.objective(rec, obs)


def test_gradient_matches_finite_differences():
    nsteps = 45
    p_true, *_ = _problem(sponge=(3, 0.25), vjit=0.2, seed=9, nsteps=nsteps,
                          src=[(2, 3, 2), (7, 5, 3)])
    obs, _ = p_true.forward(nsteps)
    p, *_ = _problem(sponge=(3, 0.25), vjit=0.0, seed=9, nsteps=nsteps, src=[(2, 3, 2), (7, 5, 3)])
    rec, states = p.forward(nsteps, keep_states=True)
    grad = p.gradient_m(rec - obs, states)
    m0 = p.m[R:-R, R:-R, R:-R].copy()
    g = np.random.default_rng(10)
    for _ in range(3):
        d = g.normal(size=m0.shape) * m0
        eps = 1e-4
        jp = _objective_at(m0 + eps * d, p, obs, nsteps)
        jm = _objective_at(m0 - eps * d, p, obs, nsteps)
        fd = (jp - jm) / (2 * eps)
        an = float(np.sum(grad * d))
        assert fd == pytest.approx(an, rel=1e-6)
    # Taylor remainder |J(m+e d) - J(m) - e <g, d>| shrinks as e^2.
    j0 = oracle.objective(rec, obs)
    d = g.normal(size=m0.shape) * m0
    an = float(np.sum(grad * d))
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        errs.append(abs(_objective_at(m0 + eps * d, p, obs, nsteps) - j0 - eps * an))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < s < 2.2 for s in slopes)


def test_step_at_points_equals_the_full_step():
    # The point-by-point step (used at full size, where a full FP64 step does
    # not fit the test budget) against the oracle's full-grid step.
    n = (14, 12, 13)
    prob, v, dt, h = _problem(n=n, sponge=(4, 0.05), vjit=0.2, src=[(5, 6, 4)], nsteps=4)
    g = np.random.default_rng(3)
    a_cur, a_prev = oracle.pad(g.uniform(-1, 1, n), R), oracle.pad(g.uniform(-1, 1, n), R)
    full = prob.step(a_cur, a_prev, 0, 2)
    nz, ny, nx = n
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    args = (R, oracle.fd2_star_coeffs(R), oracle.model_m(v, dt, h), (4, 0.05), (5, 6, 4))
    got = oracle.wave_step_points(*args, prob.amp[2, 0], a_cur, a_prev, pts)
    want = full[R:-R, R:-R, R:-R].ravel()
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # the source term lands on the source point only, scaled by G there
    quiet = oracle.wave_step_points(*args, 0.0, a_cur, a_prev, pts)
    src_idx = (4 * ny + 6) * nx + 5
    diff = got - quiet
    g = oracle.sponge_1d(nx, 4, 0.05)[5] * oracle.sponge_1d(ny, 4, 0.05)[6] * oracle.sponge_1d(nz, 4, 0.05)[4]
    assert prob.amp[2, 0] != 0.0 and diff[src_idx] == pytest.approx(g * prob.amp[2, 0], rel=1e-12)
    assert np.count_nonzero(diff) == 1
