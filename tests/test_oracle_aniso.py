"""Pins of the FP64 VTI and TTI oracle (oracle/aniso.py).

Each function is tied to facts fixed outside its own code: the textbook
first-derivative weights and their Fourier symbol, exactness on polynomials
(closed-form derivatives of quadratic fields, where every term of the
coupled right-hand sides has a distinct value), and reductions to the
acoustic step of oracle.c (isotropic media).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import aniso
import workloads


# ------------------------------------------------------------ weights

def test_fd1_weights_closed_forms():
    assert aniso.fd1_weights(1) == [Fraction(1, 2)]
    assert aniso.fd1_weights(2) == [Fraction(2, 3), Fraction(-1, 12)]
    assert aniso.fd1_weights(3) == [Fraction(3, 4), Fraction(-3, 20), Fraction(1, 60)]
    assert aniso.fd1_weights(4) == [Fraction(4, 5), Fraction(-1, 5), Fraction(4, 105), Fraction(-1, 280)]


def test_workload_fd8_rows_are_the_exact_weights():
    w2, w1 = workloads.fd8_rows()
    np.testing.assert_allclose(w2, aniso.fd2_row(4).astype(np.float32), rtol=0, atol=0)
    np.testing.assert_allclose(w1, aniso.fd1_row(4).astype(np.float32), rtol=0, atol=0)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_fd1_row_is_exact_to_order_2r(r):
    row = aniso.fd1_row(r)
    d = np.arange(-r, r + 1, dtype=np.float64)
    assert np.allclose(row, -row[::-1])
    for p in range(0, 2 * r + 1):                     # d/dx x^p at 0
        assert math.isclose(float(row @ d ** p), 1.0 if p == 1 else 0.0, abs_tol=1e-12)
    assert abs(float(row @ d ** (2 * r + 1))) > 1e-3  # order exactly 2r
    # Fourier symbol: sum_k b_k 2 sin(k w) = w + O(w^{2r+1})
    w = 1e-2
    sym = sum(float(row[r + k]) * 2 * math.sin(k * w) for k in range(1, r + 1))
    assert abs(sym - w) < 10 * w ** (2 * r + 1) + 1e-15


# ------------------------------------------------------------ fields

def _coords(n, r):
    nz, ny, nx = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def _padded(f, r):
    return oracle.pad(f, r)


def _deep(n, r):
    """Mask of interior points whose radius-r neighbourhood (all axes) is interior."""
    nz, ny, nx = n
    m = np.zeros(n, bool)
    m[r:nz - r, r:ny - r, r:nx - r] = True
    return m


N = (12, 13, 14)


@pytest.mark.parametrize("r", [1, 2, 4])
def test_second_derivatives_exact_on_quadratics(r):
    x, y, z = _coords(N, r)
    deep = _deep(N, r)
    for f, want in [
        (x * x, dict(xx=2, yy=0, zz=0, xy=0, xz=0, yz=0)),
        (x * z, dict(xx=0, yy=0, zz=0, xy=0, xz=1, yz=0)),
        (y * z + 3 * x * y, dict(xx=0, yy=0, zz=0, xy=3, xz=0, yz=1)),
        (z * z - y * y + 0.5 * x * y * 2, dict(xx=0, yy=-2, zz=2, xy=1, xz=0, yz=0)),
    ]:
        d = aniso.second_derivatives(r, _padded(f, r))
        for k, v in want.items():
            np.testing.assert_allclose(d[k][deep], v, atol=1e-9, err_msg=k)


def test_mixed_derivative_is_the_tensor_product_stencil():
    # brute force on a small random field: d_xz f = sum_ij b_i b_j f(x+i, z+j)
    r = 2
    g = np.random.default_rng(3)
    f = g.uniform(-1, 1, size=(7, 6, 8))
    fp = _padded(f, r)
    row = aniso.fd1_row(r)
    d = aniso.second_derivatives(r, fp)
    want = np.zeros_like(f)
    for z in range(7):
        for y in range(6):
            for x in range(8):
                s = 0.0
                for i in range(-r, r + 1):
                    for j in range(-r, r + 1):
                        s += row[i + r] * row[j + r] * fp[z + r + j, y + r, x + r + i]
                want[z, y, x] = s
    np.testing.assert_allclose(d["xz"], want, rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------ VTI

def _vti_medium(n, seed=0):
    g = np.random.default_rng(seed)
    vp = 2000.0 * (1 + 0.2 * g.uniform(-1, 1, size=n))
    eps = g.uniform(0.0, 0.3, size=n)
    delta = g.uniform(-0.1, 0.2, size=n)
    h, dt = 10.0, 0.3 * 10.0 / 2400.0 / math.sqrt(1.6)
    return vp, eps, delta, dt, h


def test_vti_medium_closed_form():
    mh, mv = aniso.vti_medium(2000.0, 0.25, 0.04, 1e-3, 10.0)
    m = 2000.0 ** 2 * 1e-6 / 100.0
    assert mh == pytest.approx(m * 1.5, rel=1e-15)
    assert mv == pytest.approx(m * math.sqrt(1.08), rel=1e-15)


@pytest.mark.parametrize("r", [2, 4])
def test_vti_quadratic_fields_pin_every_coupling(r):
    # sigma_H = x^2 + y^2, sigma_V = z^2: (dxx + dyy) sigma_H = 4, dzz sigma_V = 2,
    # (dxx + dyy) sigma_V = 0, dzz sigma_H = 0; then the fields swapped.
    x, y, z = _coords(N, r)
    vp, eps, delta, dt, h = _vti_medium(N)
    mh, mv = aniso.vti_medium(vp, eps, delta, dt, h)
    deep = _deep(N, r)
    c = oracle.fd2_star_coeffs(r)
    zero = np.zeros_like(_padded(x, r))
    a, b = x * x + y * y, z * z
    h1, v1 = aniso.vti_step(r, c, mh, mv, None, None, 0.0, _padded(a, r), _padded(b, r), zero, zero)
    np.testing.assert_allclose(h1[r:-r, r:-r, r:-r][deep], (2 * a + 4 * mh + 2 * mv)[deep], rtol=1e-12)
    np.testing.assert_allclose(v1[r:-r, r:-r, r:-r][deep], (2 * b)[deep], rtol=1e-12)
    h2, v2 = aniso.vti_step(r, c, mh, mv, None, None, 0.0, _padded(b, r), _padded(a, r), zero, zero)
    np.testing.assert_allclose(h2[r:-r, r:-r, r:-r][deep], (2 * b)[deep], rtol=1e-12)
    np.testing.assert_allclose(v2[r:-r, r:-r, r:-r][deep], (2 * a + 4 * mv + 2 * mh)[deep], rtol=1e-12)


def test_vti_isotropic_equal_stresses_is_the_acoustic_step():
    r, nsteps = 4, 12
    n = (11, 10, 12)
    vp, _, _, dt, h = _vti_medium(n, seed=1)
    zeros = np.zeros(n)
    mh, mv = aniso.vti_medium(vp, zeros, zeros, dt, h)
    c = oracle.fd2_star_coeffs(r)
    amp = np.zeros((nsteps, 1))
    amp[:, 0] = dt * dt * workloads.ricker(np.arange(nsteps) * dt, 60.0, 1.0 / 60.0) * 1e6
    src = (5, 4, 6)
    ac = oracle.WaveProblem(r, c, oracle.model_m(vp, dt, h), (3, 0.1), [src], amp, zrec=1)
    a_prev, a_cur = ac.zeros(), ac.zeros()
    sh_p, sh, sv_p, sv = ac.zeros(), ac.zeros(), ac.zeros(), ac.zeros()
    for k in range(nsteps):
        a_next = ac.step(a_cur, a_prev, 0, k)
        sh_n, sv_n = aniso.vti_step(r, c, mh, mv, (3, 0.1), src, amp[k, 0], sh, sv, sh_p, sv_p)
        a_prev, a_cur = a_cur, a_next
        sh_p, sh, sv_p, sv = sh, sh_n, sv, sv_n
        scale = np.abs(a_cur).max()
        assert scale > 0
        np.testing.assert_allclose(sh, a_cur, rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(sv, a_cur, rtol=0, atol=1e-12 * scale)


def test_vti_points_equal_the_full_step():
    r = 3
    n = (9, 11, 10)
    g = np.random.default_rng(4)
    vp, eps, delta, dt, h = _vti_medium(n, seed=2)
    mh, mv = aniso.vti_medium(vp, eps, delta, dt, h)
    c = workloads.normal_coeffs("star", r, workload=4)
    f = [_padded(g.uniform(-1, 1, size=n), r) for _ in range(4)]
    src = (3, 4, 5)
    full = aniso.vti_step(r, c, mh, mv, (2, 0.2), src, 0.7, *f)
    pts = np.array([[x, y, z] for z in range(n[0]) for y in range(n[1]) for x in range(n[2])][::7])
    pts = np.vstack([pts, [src]])
    ph, pv = aniso.vti_step_points(r, c, mh, mv, (2, 0.2), src, 0.7, *f, pts)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    np.testing.assert_allclose(ph, full[0][z + r, y + r, x + r], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(pv, full[1][z + r, y + r, x + r], rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------ TTI

def _tti_medium(n, seed=0):
    g = np.random.default_rng(seed)
    vp = 2000.0 * (1 + 0.2 * g.uniform(-1, 1, size=n))
    vs = 0.4 * vp * (1 + 0.1 * g.uniform(-1, 1, size=n))
    eps = g.uniform(0.0, 0.3, size=n)
    delta = g.uniform(-0.1, 0.2, size=n)
    alpha = g.uniform(0.5, 1.5, size=n)
    th = g.uniform(0, math.pi / 2, size=n)
    ph = g.uniform(-math.pi, math.pi, size=n)
    h, dt = 10.0, 1e-3
    return aniso.tti_medium(vp, vs, eps, delta, alpha, dt, h), aniso.tilt_axis(th, ph)


def test_tilt_axis_is_a_unit_vector_giving_the_printed_coefficients():
    g = np.random.default_rng(0)
    th, ph = g.uniform(0, math.pi, 50), g.uniform(-math.pi, math.pi, 50)
    nx, ny, nz = aniso.tilt_axis(th, ph)
    np.testing.assert_allclose(nx * nx + ny * ny + nz * nz, 1.0, rtol=1e-14)
    s, c = np.sin, np.cos
    np.testing.assert_allclose(nx * nx, s(th) ** 2 * c(ph) ** 2, atol=1e-15)
    np.testing.assert_allclose(ny * ny, s(th) ** 2 * s(ph) ** 2, atol=1e-15)
    np.testing.assert_allclose(nz * nz, c(th) ** 2, atol=1e-15)
    np.testing.assert_allclose(2 * nx * ny, s(th) ** 2 * s(2 * ph), atol=1e-15)
    np.testing.assert_allclose(2 * ny * nz, s(2 * th) * s(ph), atol=1e-15)
    np.testing.assert_allclose(2 * nx * nz, s(2 * th) * c(ph), atol=1e-15)


@pytest.mark.parametrize("r", [2, 4])
def test_h1_of_a_squared_projection(r):
    # f = (n0 . x)^2 with a fixed unit n0: H1 f = 2 (n . n0)^2 for the
    # per-point axis n, and H2 f = 2 - H1 f
    x, y, z = _coords(N, r)
    _, n = _tti_medium(N, seed=5)
    n0 = np.array([0.3, -0.5, 0.8])
    n0 /= np.linalg.norm(n0)
    f = (n0[0] * x + n0[1] * y + n0[2] * z) ** 2
    d = aniso.second_derivatives(r, _padded(f, r))
    deep = _deep(N, r)
    dot = n[0] * n0[0] + n[1] * n0[1] + n[2] * n0[2]
    got = aniso.h1(n, d)
    np.testing.assert_allclose(got[deep], (2 * dot * dot)[deep], atol=1e-9)
    lap = d["xx"] + d["yy"] + d["zz"]
    np.testing.assert_allclose(lap[deep], 2.0, atol=1e-9)


@pytest.mark.parametrize("r", [2, 4])
def test_tti_quadratic_fields_pin_every_term(r):
    # Constant tilt n: for u = (n . x)^2, H1 u = 2, H2 u = 0; for w = |x|^2,
    # H1 w = 2, H2 w = 4.  Each right-hand side term then has its own value.
    x, y, z = _coords(N, r)
    med, _ = _tti_medium(N, seed=6)
    vpx2, vpz2, vpn2, vsz2, al = med
    th, ph = 0.7, -1.1
    n = tuple(np.full(N, v) for v in aniso.tilt_axis(th, ph))
    u = (n[0] * x + n[1] * y + n[2] * z) ** 2
    w = x * x + y * y + z * z
    deep = _deep(N, r)
    zero = np.zeros_like(_padded(x, r))
    for p, q, h1p, h2p, h1q, h2q in [(u, w, 2, 0, 2, 4), (w, u, 2, 4, 2, 0), (u, u, 2, 0, 2, 0)]:
        p1, q1 = aniso.tti_step(r, med, n, None, None, 0.0, _padded(p, r), _padded(q, r), zero, zero)
        rp = vpx2 * h2p + al * vpz2 * h1q + vsz2 * (h1p - al * h1q)
        rq = vpn2 / al * h2p + vpz2 * h1q - vsz2 * (h2p / al - h2q)
        np.testing.assert_allclose(p1[r:-r, r:-r, r:-r][deep], (2 * p + rp)[deep], rtol=1e-9)
        np.testing.assert_allclose(q1[r:-r, r:-r, r:-r][deep], (2 * q + rq)[deep], rtol=1e-9)


def test_tti_isotropic_is_the_acoustic_step():
    # alpha = 1, vsz = 0, vpx = vpz = vpn = v, p = q: both obey the acoustic
    # step with m = v^2 dt^2 / h^2, whatever the tilt
    r, nsteps = 4, 10
    n = (11, 12, 10)
    g = np.random.default_rng(8)
    v = 2000.0 * (1 + 0.2 * g.uniform(-1, 1, size=n))
    h, dt = 10.0, 0.3 * 10.0 / 2400.0
    zeros = np.zeros(n)
    med = aniso.tti_medium(v, zeros, zeros, zeros, np.ones(n), dt, h)
    tilt = aniso.tilt_axis(g.uniform(0, math.pi, n), g.uniform(-math.pi, math.pi, n))
    c = oracle.fd2_star_coeffs(r)
    amp = np.zeros((nsteps, 1))
    amp[:, 0] = dt * dt * workloads.ricker(np.arange(nsteps) * dt, 60.0, 1.0 / 60.0) * 1e6
    src = (4, 5, 6)
    ac = oracle.WaveProblem(r, c, oracle.model_m(v, dt, h), (3, 0.1), [src], amp, zrec=1)
    a_prev, a_cur = ac.zeros(), ac.zeros()
    p_p, p, q_p, q = ac.zeros(), ac.zeros(), ac.zeros(), ac.zeros()
    for k in range(nsteps):
        a_next = ac.step(a_cur, a_prev, 0, k)
        p_n, q_n = aniso.tti_step(r, med, tilt, (3, 0.1), src, amp[k, 0], p, q, p_p, q_p)
        a_prev, a_cur = a_cur, a_next
        p_p, p, q_p, q = p, p_n, q, q_n
        scale = np.abs(a_cur).max()
        np.testing.assert_allclose(p, a_cur, rtol=0, atol=1e-11 * scale)
        np.testing.assert_allclose(q, a_cur, rtol=0, atol=1e-11 * scale)


def test_tti_points_equal_the_full_step():
    r = 3
    n = (9, 11, 10)
    g = np.random.default_rng(12)
    med, tilt = _tti_medium(n, seed=3)
    f = [_padded(g.uniform(-1, 1, size=n), r) for _ in range(4)]
    src = (4, 5, 3)
    full = aniso.tti_step(r, med, tilt, (2, 0.2), src, 0.9, *f)
    pts = np.array([[x, y, z] for z in range(n[0]) for y in range(n[1]) for x in range(n[2])][::5])
    pts = np.vstack([pts, [src]])
    pp, pq = aniso.tti_step_points(r, med, tilt, (2, 0.2), src, 0.9, *f, pts)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    np.testing.assert_allclose(pp, full[0][z + r, y + r, x + r], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pq, full[1][z + r, y + r, x + r], rtol=1e-12, atol=1e-12)
