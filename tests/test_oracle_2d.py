"""Pins of the oracle's planar stencils (Table I's 2D kernels): a library
correlation, the 3D oracle with its z weights zeroed, polynomial exactness of
the FD Laplacian, and the point-wise variant."""
import numpy as np
import pytest
from scipy import ndimage

import oracle
import workloads


@pytest.mark.parametrize("shape", ["star2d", "box2d"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_planar_matches_scipy_correlate(shape, r):
    g = np.random.default_rng(r).uniform(-1, 1, (3, 17 + 2 * r, 21 + 2 * r))
    c = workloads.normal_coeffs(shape, r, workload=9, salt=r).astype(np.float64)
    w = 2 * r + 1
    if shape == "box2d":
        k = c.reshape(w, w)
    else:
        k = np.zeros((w, w))
        k[r, :] += c[0]
        k[:, r] += c[1]
    got = oracle.stencil2d(shape, r, c, g)
    for z in range(g.shape[0]):
        ref = ndimage.correlate(g[z], k, mode="constant")[r:-r, r:-r]
        assert np.abs(got[z] - ref).max() <= 1e-12


@pytest.mark.parametrize("shape", ["star2d", "box2d"])
@pytest.mark.parametrize("r", [1, 3])
def test_planar_equals_3d_oracle_without_z(shape, r):
    g = np.random.default_rng(10 + r).uniform(-1, 1, (4, 12 + 2 * r, 15 + 2 * r))
    c = workloads.normal_coeffs(shape, r, workload=9, salt=20 + r).astype(np.float64)
    w = 2 * r + 1
    if shape == "box2d":
        c3 = np.zeros((w, w, w))
        c3[r] = c.reshape(w, w)
        s3 = "box"
    else:
        c3 = np.zeros((3, w))
        c3[:2] = c
        s3 = "star"
    padded = np.zeros((g.shape[0] + 2 * r,) + g.shape[1:])
    padded[r:-r] = g
    assert np.abs(oracle.stencil2d(shape, r, c, g) - oracle.stencil(s3, r, c3, padded)).max() <= 1e-12


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_planar_fd_laplacian_is_exact_on_polynomials(r):
    # star2d with the exact FD weights on both axes reproduces the 2D
    # Laplacian of every polynomial of degree <= 2r+1 per axis
    c = np.asarray(oracle.fd2_star_coeffs(r), dtype=np.float64)[:2].reshape(-1)   # x and y lines
    n = 9
    y, x = np.meshgrid(np.arange(n + 2 * r) - r, np.arange(n + 2 * r) - r, indexing="ij")
    for p in range(2 * r + 2):
        for q in range(2 * r + 2 - p):
            u = (0.3 * x) ** p * (0.2 * y) ** q
            lap = np.zeros_like(u)
            if p >= 2:
                lap += p * (p - 1) * 0.09 * (0.3 * x) ** (p - 2) * (0.2 * y) ** q
            if q >= 2:
                lap += q * (q - 1) * 0.04 * (0.3 * x) ** p * (0.2 * y) ** (q - 2)
            got = oracle.stencil2d("star2d", r, c, u[None])[0]
            assert np.abs(got - lap[r:-r, r:-r]).max() <= 1e-9 * max(1.0, np.abs(lap).max())


@pytest.mark.parametrize("shape", ["star2d", "box2d"])
def test_planar_points_equal_the_full_planar_stencil(shape):
    r = 3
    g = np.random.default_rng(4).uniform(-1, 1, (2, 14 + 2 * r, 11 + 2 * r)).astype(np.float32)
    c = workloads.normal_coeffs(shape, r, workload=9, salt=7)
    full = oracle.stencil2d(shape, r, c, g)
    pts = np.array([[0, 0, 0], [10, 13, 1], [5, 7, 0], [10, 0, 1]])
    got = oracle.stencil2d_points(shape, r, c, g, pts)
    assert np.abs(got - full[pts[:, 2], pts[:, 1], pts[:, 0]]).max() <= 1e-12
