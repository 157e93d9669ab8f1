"""FP64 oracle of the coupled anisotropic wave steps (VTI and TTI media).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it.  It never imports the CUDA library.

The paper gives the continuous equations (Sec. 2.1) and no discretisation.
Both steps here use the same damped leapfrog form as the acoustic step of
``oracle.c`` -- u^{n+1} = G (2 u^n - G u^{n-1} + dt^2 RHS(u^n) + s^n) with
the Cerjan profile G and a zero halo of width r -- and high-order central
finite differences for every derivative (grid spacing h, dt^2/h^2 folded into
the medium).

VTI (Sec. 2.1, the sigma_H / sigma_V system as printed):

    sigma_H'' = Vp^2 [ (1+2 eps)(d_xx + d_yy) sigma_H + sqrt(1+2 delta) d_zz sigma_V ]
    sigma_V'' = Vp^2 [ sqrt(1+2 delta)(d_xx + d_yy) sigma_V + (1+2 eps) d_zz sigma_H ]

TTI (Sec. 2.1, the p / q system with H1 and H2, and Sec. 4.7 for the mixed
derivatives as composed first derivatives):

    p'' = vpx^2 H2 p + alpha vpz^2 H1 q + vsz^2 H1 (p - alpha q)
    q'' = vpn^2 / alpha H2 p + vpz^2 H1 q - vsz^2 H2 (p / alpha - q)
    H1  = sum_ij n_i n_j d_ij,  n = (sin th cos ph, sin th sin ph, cos th)
    H2  = d_xx + d_yy + d_zz - H1

Second derivatives along one axis use the radius-r central weights; a mixed
derivative d_ij (i != j) is the radius-r central first derivative along j
followed by the one along i, both on the zero-padded field.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from . import fd2_weights, sponge_1d, stencil, stencil_points


# ------------------------------------------------------------ FD weights

def fd1_weights(r: int) -> list:
    """Central first-derivative weights b_1..b_r of radius r (exact
    rationals): the antisymmetric stencil sum_k b_k (f(k) - f(-k)) must give
    f'(0) on x, x^3, ..., x^{2r-1}:  2 sum_k b_k k^{2j-1} = delta_{j,1}."""
    n = r
    M = [[Fraction(2 * k ** (2 * j - 1)) for k in range(1, n + 1)] + [Fraction(1 if j == 1 else 0)]
         for j in range(1, n + 1)]
    for col in range(n):
        piv = next(i for i in range(col, n) if M[i][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [v / pv for v in M[col]]
        for i in range(n):
            if i != col and M[i][col] != 0:
                f = M[i][col]
                M[i] = [vi - f * vc for vi, vc in zip(M[i], M[col])]
    return [M[i][n] for i in range(n)]


def fd1_row(r: int) -> np.ndarray:
    """The first-derivative weights as a row over offsets -r..r (FP64)."""
    b = fd1_weights(r)
    return np.array([-float(b[-d - 1]) if d < 0 else (0.0 if d == 0 else float(b[d - 1]))
                     for d in range(-r, r + 1)])


# ------------------------------------------------------------ helpers

def _damping(shape, sponge):
    nz, ny, nx = shape
    if sponge is None:
        return np.ones(shape)
    w, a = sponge
    return (sponge_1d(nz, w, a)[:, None, None] * sponge_1d(ny, w, a)[None, :, None]
            * sponge_1d(nx, w, a)[None, None, :])


def _axes(coeffs, keep):
    """Star weights with only the axes in `keep` (0 = x, 1 = y, 2 = z)."""
    c = np.array(np.asarray(coeffs, dtype=np.float64).reshape(3, -1))
    for a in range(3):
        if a not in keep:
            c[a] = 0.0
    return c


def _interior(f, r):
    return np.asarray(f, dtype=np.float64)[r:-r, r:-r, r:-r]


def _source(shape, src, s_amp):
    s = np.zeros(shape)
    if src is not None and src[0] >= 0:
        s[src[2], src[1], src[0]] = float(s_amp)
    return s


def _leapfrog(r, g, cur, prev, rhs, s):
    """Padded u^{n+1} = G (2 u^n - G u^{n-1} + rhs + s), zero halo."""
    out = np.zeros(np.asarray(cur).shape)
    out[r:-r, r:-r, r:-r] = g * (2.0 * _interior(cur, r) - g * _interior(prev, r) + rhs + s)
    return out


# ------------------------------------------------------------ VTI

def vti_medium(vp, eps, delta, dt: float, h: float):
    """(mh, mv) = (m (1 + 2 eps), m sqrt(1 + 2 delta)), m = vp^2 dt^2 / h^2:
    the two coefficients of the VTI system, per interior point (FP64)."""
    vp = np.asarray(vp, np.float64)
    m = vp * vp * (float(dt) * float(dt)) / (float(h) * float(h))
    return (m * (1.0 + 2.0 * np.asarray(eps, np.float64)),
            m * np.sqrt(1.0 + 2.0 * np.asarray(delta, np.float64)))


def vti_step(r, coeffs, mh, mv, sponge, src, s_amp, sh_cur, sv_cur, sh_prev, sv_prev):
    """One VTI step of one shot: padded (sigma_H, sigma_V)^{n+1}.

    coeffs: (3, 2r+1) unscaled second-derivative weights per axis; mh, mv:
    interior coefficient fields of ``vti_medium``; the source s^n is added to
    both stresses at `src` (x, y, z)."""
    r = int(r)
    lh = lambda f: stencil("star", r, _axes(coeffs, (0, 1)), f)   # (d_xx + d_yy)
    lz = lambda f: stencil("star", r, _axes(coeffs, (2,)), f)     # d_zz
    mh = np.asarray(mh, np.float64)
    mv = np.asarray(mv, np.float64)
    g = _damping(mh.shape, sponge)
    s = _source(mh.shape, src, s_amp)
    rhs_h = mh * lh(sh_cur) + mv * lz(sv_cur)
    rhs_v = mv * lh(sv_cur) + mh * lz(sh_cur)
    return (_leapfrog(r, g, sh_cur, sh_prev, rhs_h, s), _leapfrog(r, g, sv_cur, sv_prev, rhs_v, s))


def vti_step_points(r, coeffs, mh, mv, sponge, src, s_amp, sh_cur, sv_cur, sh_prev, sv_prev, xyz):
    """The VTI step at interior points ``xyz`` (npts, 3) only (fields read in
    place, FP32 or FP64): returns (sigma_H^{n+1}, sigma_V^{n+1}) there."""
    r = int(r)
    pts = np.ascontiguousarray(np.asarray(xyz, dtype=np.int64).reshape(-1, 3))
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    cxy, cz = _axes(coeffs, (0, 1)), _axes(coeffs, (2,))
    mh = np.asarray(mh)[z, y, x].astype(np.float64)
    mv = np.asarray(mv)[z, y, x].astype(np.float64)
    nz, ny, nx = np.asarray(sh_cur).shape
    nz, ny, nx = nz - 2 * r, ny - 2 * r, nx - 2 * r
    if sponge is None:
        g = np.ones(len(pts))
    else:
        g = sponge_1d(nx, *sponge)[x] * sponge_1d(ny, *sponge)[y] * sponge_1d(nz, *sponge)[z]
    s = np.where((x == src[0]) & (y == src[1]) & (z == src[2]), float(s_amp), 0.0)

    def at(f):
        return np.asarray(f)[z + r, y + r, x + r].astype(np.float64)

    rhs_h = mh * stencil_points("star", r, cxy, sh_cur, pts) + mv * stencil_points("star", r, cz, sv_cur, pts)
    rhs_v = mv * stencil_points("star", r, cxy, sv_cur, pts) + mh * stencil_points("star", r, cz, sh_cur, pts)
    return (g * (2.0 * at(sh_cur) - g * at(sh_prev) + rhs_h + s),
            g * (2.0 * at(sv_cur) - g * at(sv_prev) + rhs_v + s))


# ------------------------------------------------------------ TTI

def tti_medium(vp, vs, eps, delta, alpha, dt: float, h: float):
    """The velocity fields of the TTI system scaled by dt^2/h^2, from the
    usual Thomsen parameters: vpz = vp, vpx = vp sqrt(1 + 2 eps),
    vpn = vp sqrt(1 + 2 delta), vsz = vs; alpha as given.  Returns
    (vpx2, vpz2, vpn2, vsz2, alpha) (FP64, interior)."""
    k = float(dt) * float(dt) / (float(h) * float(h))
    vp2 = np.asarray(vp, np.float64) ** 2 * k
    return (vp2 * (1.0 + 2.0 * np.asarray(eps, np.float64)), vp2,
            vp2 * (1.0 + 2.0 * np.asarray(delta, np.float64)),
            np.asarray(vs, np.float64) ** 2 * k, np.asarray(alpha, np.float64))


def tilt_axis(theta, phi):
    """n = (sin th cos ph, sin th sin ph, cos th): H1 = (n . grad)^2 with the
    coefficients printed in Sec. 2.1."""
    th = np.asarray(theta, np.float64)
    ph = np.asarray(phi, np.float64)
    return np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)


def fd2_row(r: int) -> np.ndarray:
    """The second-derivative weights as a row over offsets -r..r (FP64)."""
    w = fd2_weights(r)
    return np.array([float(w[abs(d)]) for d in range(-r, r + 1)])


def second_derivatives(r, f, row2=None, row1=None):
    """The six second derivatives of padded field f on its interior:
    dict with keys xx, yy, zz, xy, xz, yz (FP64).  Axis ones use the
    second-derivative row `row2` (offsets -r..r; default the radius-r
    central weights); mixed ones compose two first derivatives of row `row1`
    (default the radius-r central weights) on the zero-padded field
    (Sec. 4.7)."""
    r = int(r)
    row2 = fd2_row(r) if row2 is None else np.asarray(row2, np.float64).reshape(-1)
    row1 = fd1_row(r) if row1 is None else np.asarray(row1, np.float64).reshape(-1)
    f = np.asarray(f, np.float64)
    zero = np.zeros(2 * r + 1)
    out = {}
    for name, axis in (("xx", 0), ("yy", 1), ("zz", 2)):
        c = np.array([zero, zero, zero])
        c[axis] = row2
        out[name] = stencil("star", r, c, f)

    def d1(g, axis):   # first derivative along `axis`, padded with a zero halo
        c = np.array([zero, zero, zero])
        c[axis] = row1
        res = np.zeros_like(g)
        res[r:-r, r:-r, r:-r] = stencil("star", r, c, g)
        return res

    # The inner derivative vanishes in the halo (the field is zero there, and
    # the inner axis does not leave it), so composing on the interior and
    # zero-padding equals the tensor-product stencil on the zero-padded field.
    for name, (a, b) in (("xy", (0, 1)), ("xz", (0, 2)), ("yz", (1, 2))):
        outer_c = np.array([zero, zero, zero])
        outer_c[a] = row1
        out[name] = stencil("star", r, outer_c, d1(f, b))
    return out


def h1(n, d):
    """H1 of Sec. 2.1 from the six second derivatives d and the tilt axis n."""
    nx, ny, nz = n
    return (nx * nx * d["xx"] + ny * ny * d["yy"] + nz * nz * d["zz"]
            + 2.0 * nx * ny * d["xy"] + 2.0 * ny * nz * d["yz"] + 2.0 * nx * nz * d["xz"])


def tti_step(r, medium, n, sponge, src, s_amp, p_cur, q_cur, p_prev, q_prev, row2=None, row1=None):
    """One TTI step of one shot: padded (p, q)^{n+1}.

    medium: (vpx2, vpz2, vpn2, vsz2, alpha) of ``tti_medium`` (interior);
    n: the tilt axis (nx, ny, nz) of ``tilt_axis`` (interior fields);
    row2, row1: derivative weights as in ``second_derivatives``."""
    r = int(r)
    vpx2, vpz2, vpn2, vsz2, alpha = (np.asarray(a, np.float64) for a in medium)
    dp = second_derivatives(r, p_cur, row2, row1)
    dq = second_derivatives(r, q_cur, row2, row1)
    h1p, h1q = h1(n, dp), h1(n, dq)
    h2p = dp["xx"] + dp["yy"] + dp["zz"] - h1p
    h2q = dq["xx"] + dq["yy"] + dq["zz"] - h1q
    rhs_p = vpx2 * h2p + alpha * vpz2 * h1q + vsz2 * (h1p - alpha * h1q)
    rhs_q = vpn2 / alpha * h2p + vpz2 * h1q - vsz2 * (h2p / alpha - h2q)
    g = _damping(vpx2.shape, sponge)
    s = _source(vpx2.shape, src, s_amp)
    return (_leapfrog(r, g, p_cur, p_prev, rhs_p, s), _leapfrog(r, g, q_cur, q_prev, rhs_q, s))


def tti_step_points(r, medium, n, sponge, src, s_amp, p_cur, q_cur, p_prev, q_prev, xyz, row2=None, row1=None):
    """The TTI step at interior points ``xyz`` (npts, 3) only: returns
    (p^{n+1}, q^{n+1}) there.  medium, n: full interior fields as in
    ``tti_step`` (indexed at the points); fields read in place (FP32 or
    FP64, zero halo).  Each derivative is the same sum as in
    ``second_derivatives``, gathered point by point."""
    r = int(r)
    row2 = fd2_row(r) if row2 is None else np.asarray(row2, np.float64).reshape(-1)
    row1 = fd1_row(r) if row1 is None else np.asarray(row1, np.float64).reshape(-1)
    pts = np.ascontiguousarray(np.asarray(xyz, dtype=np.int64).reshape(-1, 3))
    x, y, z = pts[:, 0] + r, pts[:, 1] + r, pts[:, 2] + r       # padded indices
    offs = range(-r, r + 1)

    def derivs(f):
        f = np.asarray(f)
        at = lambda dx, dy, dz: f[z + dz, y + dy, x + dx].astype(np.float64)
        d = {"xx": sum(row2[i + r] * at(i, 0, 0) for i in offs),
             "yy": sum(row2[i + r] * at(0, i, 0) for i in offs),
             "zz": sum(row2[i + r] * at(0, 0, i) for i in offs),
             "xy": sum(row1[i + r] * row1[j + r] * at(i, j, 0) for i in offs for j in offs),
             "xz": sum(row1[i + r] * row1[j + r] * at(i, 0, j) for i in offs for j in offs),
             "yz": sum(row1[i + r] * row1[j + r] * at(0, i, j) for i in offs for j in offs)}
        return d

    px, py_, pz = pts[:, 0], pts[:, 1], pts[:, 2]
    take = lambda a: np.asarray(a)[pz, py_, px].astype(np.float64)
    vpx2, vpz2, vpn2, vsz2, alpha = (take(a) for a in medium)
    nn = tuple(take(c) for c in n)
    dp, dq = derivs(p_cur), derivs(q_cur)
    h1p, h1q = h1(nn, dp), h1(nn, dq)
    h2p = dp["xx"] + dp["yy"] + dp["zz"] - h1p
    h2q = dq["xx"] + dq["yy"] + dq["zz"] - h1q
    rhs_p = vpx2 * h2p + alpha * vpz2 * h1q + vsz2 * (h1p - alpha * h1q)
    rhs_q = vpn2 / alpha * h2p + vpz2 * h1q - vsz2 * (h2p / alpha - h2q)
    nz_, ny_, nx_ = np.asarray(p_cur).shape
    nz_, ny_, nx_ = nz_ - 2 * r, ny_ - 2 * r, nx_ - 2 * r
    if sponge is None:
        g = np.ones(len(pts))
    else:
        g = sponge_1d(nx_, *sponge)[px] * sponge_1d(ny_, *sponge)[py_] * sponge_1d(nz_, *sponge)[pz]
    s = np.where((px == src[0]) & (py_ == src[1]) & (pz == src[2]), float(s_amp), 0.0)
    at0 = lambda f: np.asarray(f)[z, y, x].astype(np.float64)
    return (g * (2.0 * at0(p_cur) - g * at0(p_prev) + rhs_p + s),
            g * (2.0 * at0(q_cur) - g * at0(q_prev) + rhs_q + s))
