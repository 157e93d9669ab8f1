"""Pins of the FP64 stencil oracle against facts that do not come from it.

Every check below would fail for a plausible mistake in oracle.c: a dropped
axis or term, a wrong sign or offset, a transposed coefficient index, a
wrong halo origin.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import ndimage

import oracle
import workloads

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def closed_form_fd2(r):
    """Closed form of the central 2nd-derivative weights of radius r
    (Fornberg 1988): c_k = 2 (-1)^{k+1} (r!)^2 / (k^2 (r-k)! (r+k)!), k >= 1,
    and c_0 = -2 sum_k c_k."""
    ck = [Fraction(2 * (-1) ** (k + 1) * math.factorial(r) ** 2,
                   k * k * math.factorial(r - k) * math.factorial(r + k)) for k in range(1, r + 1)]
    return [-2 * sum(ck)] + ck


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_fd2_weights_closed_form(r):
    assert oracle.fd2_weights(r) == closed_form_fd2(r)


def test_fd8_weights_literal_values():
    # The radius-4 weights the 64^3 and 1024^3 workloads use.
    w = oracle.fd2_weights(4)
    assert w == [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315),
                 Fraction(-1, 560)]
    assert np.array_equal(np.float32(workloads.FD8), np.float32([float(v) for v in w]))


def test_fd8_symbol_at_nyquist():
    # 1D symbol c_0 + 2 sum_k c_k cos(k pi) at the Nyquist wavenumber is
    # exactly -2048/315 = -6.5015873...; it fixes the leapfrog CFL bound
    # v dt / h <= 2 / sqrt(3 * 2048/315) = 0.45286 for the 3D star.
    w = oracle.fd2_weights(4)
    s = w[0] + 2 * sum(w[k] * (-1) ** k for k in range(1, 5))
    assert s == Fraction(-2048, 315)


def _poly_grid(r, n, deg, seed):
    """Padded grid of p(x,y,z) = sum a_ijk x^i y^j z^k (i,j,k <= deg) and its
    exact Laplacian on the interior (numpy.polynomial, h = 1)."""
    g = np.random.default_rng(seed)
    A = g.uniform(-1, 1, size=(deg + 1, deg + 1, deg + 1))
    # coordinates centred near 0 keep round-off small
    c = (np.arange(n + 2 * r) - (n + 2 * r - 1) / 2.0) / 4.0
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")  # (x, y, z)
    P = np.polynomial.polynomial.polyval3d(X, Y, Z, A)
    lap = (np.polynomial.polynomial.polyval3d(X, Y, Z, np.polynomial.polynomial.polyder(A, 2, axis=0))
           + np.polynomial.polynomial.polyval3d(X, Y, Z, np.polynomial.polynomial.polyder(A, 2, axis=1))
           + np.polynomial.polynomial.polyval3d(X, Y, Z, np.polynomial.polynomial.polyder(A, 2, axis=2)))
    # grid spacing 1/4 -> scale the exact second derivative to unit spacing
    lap = lap / 16.0
    # (x, y, z) -> (z, y, x)
    return np.transpose(P, (2, 1, 0)).copy(), np.transpose(lap, (2, 1, 0))[r:-r, r:-r, r:-r]


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_star_polynomial_exactness(r):
    # The radius-r weights differentiate polynomials of degree <= 2r+1
    # exactly; the star applies them on all three axes (Laplacian).
    grid, lap = _poly_grid(r, 6, 2 * r + 1, seed=r)
    out = oracle.stencil("star", r, oracle.fd2_star_coeffs(r), grid)
    scale = np.abs(lap).max()
    assert np.abs(out - lap).max() <= 1e-10 * scale


@pytest.mark.parametrize("r", [1, 2, 3])
def test_star_polynomial_degree_beyond_order_fails(r):
    # Degree 2r+2 is NOT reproduced: the exactness test has teeth.
    grid, lap = _poly_grid(r, 6, 2 * r + 2, seed=10 + r)
    out = oracle.stencil("star", r, oracle.fd2_star_coeffs(r), grid)
    assert np.abs(out - lap).max() > 1e-6 * np.abs(lap).max()


def _cos_grid(shape_int, r, k, phi):
    nz, ny, nx = shape_int
    Z, Y, X = np.meshgrid(np.arange(nz + 2 * r), np.arange(ny + 2 * r), np.arange(nx + 2 * r),
                          indexing="ij")
    return Z, Y, X, np.cos(k[0] * X + k[1] * Y + k[2] * Z + phi)


@pytest.mark.parametrize("shape,r", [("star", 1), ("star", 4), ("box", 1), ("box", 2), ("box", 3)])
def test_fourier_symbol(shape, r):
    # in = cos(k.x + phi)  ->  out = Re(sigma(k) e^{i(k.x + phi)}),
    # sigma = sum_d c_d e^{i k.d}; exact on the padded grid for any weights.
    g = np.random.default_rng(100 + r)
    c = g.normal(size=oracle.n_coeffs(shape, r))
    k = g.uniform(0, math.pi, 3)
    phi = g.uniform(0, 2 * math.pi)
    Z, Y, X, grid = _cos_grid((7, 6, 9), r, k, phi)
    w = 2 * r + 1
    d = np.arange(-r, r + 1)
    if shape == "star":
        cs = c.reshape(3, w)
        sigma = sum(np.sum(cs[a] * np.exp(1j * k[a] * d)) for a in range(3))
    else:
        cb = c.reshape(w, w, w)  # [dz][dy][dx]
        DZ, DY, DX = np.meshgrid(d, d, d, indexing="ij")
        sigma = np.sum(cb * np.exp(1j * (k[0] * DX + k[1] * DY + k[2] * DZ)))
    expect = np.real(sigma * np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z + phi)))[r:-r, r:-r, r:-r]
    out = oracle.stencil(shape, r, c, grid)
    assert np.abs(out - expect).max() <= 1e-12 * max(1.0, np.abs(expect).max())


def _kernel3d(shape, r, c):
    w = 2 * r + 1
    if shape == "box":
        return np.asarray(c, np.float64).reshape(w, w, w)
    cs = np.asarray(c, np.float64).reshape(3, w)
    K = np.zeros((w, w, w))
    K[r, r, :] += cs[0]
    K[r, :, r] += cs[1]
    K[:, r, r] += cs[2]
    return K


@pytest.mark.parametrize("shape,r", [("star", 1), ("star", 2), ("star", 3), ("star", 4),
                                     ("box", 1), ("box", 2), ("box", 4)])
def test_matches_scipy_correlate(shape, r):
    # Library routine: out = correlate(in, K)[interior] with K[dz][dy][dx].
    g = np.random.default_rng(7 * r + len(shape))
    c = g.normal(size=oracle.n_coeffs(shape, r))
    grid = g.uniform(-1, 1, size=(5 + 2 * r, 11 + 2 * r, 13 + 2 * r))
    ref = ndimage.correlate(grid, _kernel3d(shape, r, c), mode="constant", cval=0.0)
    out = oracle.stencil(shape, r, c, grid)
    np.testing.assert_allclose(out, ref[r:-r, r:-r, r:-r], rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape,r", [("star", 2), ("box", 1)])
def test_brute_force_matrix_8cubed(shape, r):
    # Assemble the explicit operator column by column from unit inputs; each
    # row must hold exactly the coefficient of every neighbour, nothing else.
    n = 8
    P = n + 2 * r
    g = np.random.default_rng(3)
    c = np.round(g.normal(size=oracle.n_coeffs(shape, r)) * 64) / 64  # exact binary fractions
    K = _kernel3d(shape, r, c)
    rows = n ** 3
    M = np.zeros((rows, P ** 3))
    for j in range(P ** 3):
        e = np.zeros(P ** 3)
        e[j] = 1.0
        M[:, j] = oracle.stencil(shape, r, c, e.reshape(P, P, P)).reshape(-1)
    w = 2 * r + 1
    for (z, y, x) in [(0, 0, 0), (7, 7, 7), (3, 4, 5), (0, 7, 2)]:
        expect = np.zeros((P, P, P))
        expect[z:z + w, y:y + w, x:x + w] = K
        assert np.array_equal(M[(z * n + y) * n + x], expect.reshape(-1))


@pytest.mark.parametrize("shape,r", [("star", 4), ("box", 2)])
def test_linearity(shape, r):
    g = np.random.default_rng(11)
    c = g.normal(size=oracle.n_coeffs(shape, r))
    u = g.uniform(-1, 1, size=(6 + 2 * r,) * 3)
    w = g.uniform(-1, 1, size=(6 + 2 * r,) * 3)
    a, b = 0.37, -1.9
    lhs = oracle.stencil(shape, r, c, a * u + b * w)
    rhs = a * oracle.stencil(shape, r, c, u) + b * oracle.stencil(shape, r, c, w)
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()


def _reflect(shape, r, c):
    w = 2 * r + 1
    if shape == "box":
        return np.asarray(c).reshape(w, w, w)[::-1, ::-1, ::-1].reshape(-1)
    return np.asarray(c).reshape(3, w)[:, ::-1].reshape(-1)


@pytest.mark.parametrize("shape,r", [("star", 3), ("box", 2)])
def test_adjointness(shape, r):
    # With a zero halo, <L u, w> = <u, L^T w>, L^T having reflected weights.
    g = np.random.default_rng(5)
    c = g.normal(size=oracle.n_coeffs(shape, r))
    n = (7, 5, 6)
    u = oracle.pad(g.uniform(-1, 1, size=n), r)
    w = oracle.pad(g.uniform(-1, 1, size=n), r)
    lu = oracle.stencil(shape, r, c, u)
    ltw = oracle.stencil(shape, r, _reflect(shape, r, c), w)
    lhs = np.sum(lu * w[r:-r, r:-r, r:-r])
    rhs = np.sum(u[r:-r, r:-r, r:-r] * ltw)
    assert abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(lu * w[r:-r, r:-r, r:-r]))
    # symmetric weights are self-adjoint
    cs = 0.5 * (c + _reflect(shape, r, c))
    lu = oracle.stencil(shape, r, cs, u)
    lw = oracle.stencil(shape, r, cs, w)
    assert abs(np.sum(lu * w[r:-r, r:-r, r:-r]) - np.sum(u[r:-r, r:-r, r:-r] * lw)) <= \
        1e-13 * np.sum(np.abs(lu * w[r:-r, r:-r, r:-r]))


def test_on_axis_box_equals_star():
    r = 2
    g = np.random.default_rng(9)
    cs = g.normal(size=(3, 2 * r + 1))
    K = _kernel3d("star", r, cs)
    grid = g.uniform(-1, 1, size=(9, 8, 10))
    np.testing.assert_allclose(oracle.stencil("box", r, K.reshape(-1), grid),
                               oracle.stencil("star", r, cs, grid), rtol=0, atol=1e-13)


def test_separable_box_equals_three_1d_passes():
    r = 2
    g = np.random.default_rng(4)
    u, v, w = (g.normal(size=2 * r + 1) for _ in range(3))
    K = np.einsum("i,j,k->ijk", u, v, w)  # [dz][dy][dx]
    grid = g.uniform(-1, 1, size=(8, 9, 10))
    t = ndimage.correlate1d(grid, w, axis=2, mode="constant")
    t = ndimage.correlate1d(t, v, axis=1, mode="constant")
    t = ndimage.correlate1d(t, u, axis=0, mode="constant")
    np.testing.assert_allclose(oracle.stencil("box", r, K.reshape(-1), grid),
                               t[r:-r, r:-r, r:-r], rtol=0, atol=1e-12)


def test_seven_point_laplacian():
    # Star r=1 with [1, -2, 1] per axis is the textbook 7-point Laplacian.
    g = np.random.default_rng(2)
    f = g.uniform(-1, 1, size=(6, 7, 8))
    c = np.array([[1.0, -2.0, 1.0]] * 3)
    expect = (f[2:, 1:-1, 1:-1] + f[:-2, 1:-1, 1:-1] + f[1:-1, 2:, 1:-1] + f[1:-1, :-2, 1:-1]
              + f[1:-1, 1:-1, 2:] + f[1:-1, 1:-1, :-2] - 6 * f[1:-1, 1:-1, 1:-1])
    np.testing.assert_allclose(oracle.stencil("star", 1, c, f), expect, rtol=0, atol=1e-14)


@pytest.mark.parametrize("shape,r", [("star", 4), ("box", 2), ("box", 1)])
def test_points_match_full_sweep(shape, r):
    g = np.random.default_rng(12)
    c = g.normal(size=oracle.n_coeffs(shape, r)).astype(np.float32)
    grid = g.uniform(-1, 1, size=(7 + 2 * r, 9 + 2 * r, 11 + 2 * r)).astype(np.float32)
    full = oracle.stencil(shape, r, c, grid)
    pts = workloads.sample_points(11, 9, 7, 50, workload=1)
    for arr in (grid, grid.astype(np.float64)):
        vals = oracle.stencil_points(shape, r, c, arr, pts)
        assert np.array_equal(vals, full[pts[:, 2], pts[:, 1], pts[:, 0]])


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.stencil("box", 0, [1.0], np.zeros((3, 3, 3)))
    with pytest.raises(ValueError):
        oracle.stencil("star", 1, [1.0] * 8, np.zeros((3, 3, 3)))
    with pytest.raises(ValueError):
        oracle.stencil_points("star", 1, [1.0] * 9, np.zeros((4, 4, 4)), [[2, 0, 0]])


def test_empty_interior():
    out = oracle.stencil("star", 2, np.ones(15), np.zeros((4, 4, 4)))
    assert out.shape == (0, 0, 0)
