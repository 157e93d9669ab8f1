"""The seeded generators: determinism, shapes and the documented recipes."""
import math

import numpy as np

import workloads


def test_uniform_grid_deterministic_and_bounded():
    a = workloads.uniform_grid(9, 7, 5, 2, workload=2)
    b = workloads.uniform_grid(9, 7, 5, 2, workload=2)
    assert a.shape == (9, 11, 13) and a.dtype == np.float32
    assert np.array_equal(a, b)
    assert a.min() >= -1 and a.max() <= 1
    assert not np.array_equal(a, workloads.uniform_grid(9, 7, 5, 2, workload=3))


def test_normal_coeffs_shapes_and_scale():
    c = workloads.normal_coeffs("box", 2, workload=2)
    assert c.shape == (125,) and c.dtype == np.float32
    s = workloads.normal_coeffs("star", 3, workload=3)
    assert s.shape == (3, 7)
    big = np.concatenate([workloads.normal_coeffs("box", 4, workload=2, salt=k) for k in range(20)])
    assert abs(big.std() * math.sqrt(729) - 1.0) < 0.05


def test_sinusoid_grid_matches_direct_formula():
    r, n = 1, (6, 5, 4)
    g = workloads.sinusoid_grid(*n, r, noise=0.0, chunk=3)
    # regenerate the same parameters and evaluate sin() directly
    rg = workloads.rng(3, 0)
    a = rg.uniform(0.5, 1.0, 16)
    k = rg.uniform(0.0, math.pi / 2, size=(16, 3))
    phi = rg.uniform(0.0, 2 * math.pi, 16)
    Z, Y, X = np.meshgrid(*(np.arange(s) for s in g.shape), indexing="ij")
    ref = sum(a[j] * np.sin(k[j, 0] * X + k[j, 1] * Y + k[j, 2] * Z + phi[j]) for j in range(16))
    assert np.abs(g - ref).max() < 1e-5


def test_wave_inputs_recipe():
    w = workloads.WaveInputs(48, 40, 44, nshots=3, nsteps=30, sponge=6, noise=True)
    assert w.v.shape == (44, 40, 48) and w.v.dtype == np.float32
    assert 1500 * 0.95 <= w.v.min() and w.v.max() <= 4500 * 1.05 + 1e-3
    assert w.dt == np.float32(0.4 * 10.0 / w.vmax)
    for (x, y, z) in w.src:
        assert 6 <= x < 42 and 6 <= y < 34 and z == 6
    assert w.amp.shape == (30, 3)
    plain = workloads.WaveInputs(48, 40, 44, nshots=3, nsteps=30, sponge=6, noise=False)
    assert len(np.unique(plain.v)) == 6


def test_sample_points_cover_corners():
    p = workloads.sample_points(10, 20, 30, 100, workload=1)
    assert p.dtype == np.int64 and p.shape[1] == 3
    assert (p[:, 0] < 10).all() and (p[:, 1] < 20).all() and (p[:, 2] < 30).all()
    assert any((q == [9, 19, 29]).all() for q in p)


def test_aniso_inputs_are_seeded_and_in_range():
    import math
    a = workloads.AnisoInputs(40, 30, 50, 2, 12, tti=True)
    b = workloads.AnisoInputs(40, 30, 50, 2, 12, tti=True)
    for name in ("vp", "eps", "delta", "vs", "alpha", "theta", "phi", "amp"):
        assert np.array_equal(getattr(a, name), getattr(b, name)), name
    c = workloads.AnisoInputs(40, 30, 50, 2, 12, tti=True, salt=1)
    assert not np.array_equal(a.vp, c.vp)
    assert a.vp.shape == a.eps.shape == a.theta.shape == (50, 30, 40)
    assert 0.0 <= a.eps.min() and a.eps.max() <= 0.3
    assert -0.1 <= a.delta.min() and a.delta.max() <= 0.2
    assert np.allclose(a.vs, 0.5 * a.vp) and np.all(a.alpha == 1.0)
    assert a.theta.min() > -math.radians(15) and a.theta.max() < math.radians(60)
    # eps and delta are constant within each depth layer
    assert np.all(np.ptp(a.eps, axis=(1, 2)) == 0) and np.all(np.ptp(a.delta, axis=(1, 2)) == 0)
    # CFL 0.4 on the fastest (horizontal) speed
    vfast = float((a.vp.astype(np.float64) * np.sqrt(1 + 2 * a.eps)).max())
    assert abs(vfast * a.dt / a.h - 0.4) < 1e-6
    # first-derivative weights row: antisymmetric, the FD1_8 values
    w2, w1 = workloads.fd8_rows()
    assert np.allclose(w1, -w1[::-1]) and w1[4] == 0 and np.isclose(w1[5], 0.8)
    assert np.isclose(w2.sum(), 0.0, atol=1e-6)
