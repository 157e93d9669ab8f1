"""Seeded synthetic inputs shared, as data, by the oracle and the CUDA path.

This module generates inputs only: grids, coefficient sets, velocity models,
source wavelets and positions.  It contains none of the stencil or wave-step
arithmetic, imports neither ``oracle`` nor the CUDA package, and both sides
receive identical FP32 arrays from it.

Seeds: numpy ``default_rng(PCG64)`` with base 2507_11067 plus a workload
index (1..5 as listed in ``WORKLOADS``) plus a caller salt.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2507_11067

# The five workloads (sizes and recipes), by what they are.
WORKLOADS = {
    1: "star r=4 FD8 weights, 64^3 interior, input U[-1,1]",
    2: "box r=1 and r=2, 512^3 interior, c ~ N(0, 1/npts), input U[-1,1]",
    3: "star r=1..4, 1024^3 interior, FD8 at r=4 else N(0, 1/npts), 16 sinusoids + 1e-3 noise",
    4: "acoustic forward, 8 shots x 512^3, 500 steps, r=4 FD8, h=10, sponge 20",
    5: "acoustic gradient, 2 shots x 256^3, 200 steps, checkpoint every 20",
    6: "VTI forward, 4 shots x 512^3, r=4 FD8, layered vp with per-layer eps, delta",
    7: "TTI forward, 2 shots x 512^3, r=4 FD8 and FD1 weights, layered medium with smooth tilt",
}

# Standard 8th-order (radius-4) central second-derivative weights c_0..c_4
# (Fornberg 1988); stored as input data, checked against the oracle's exact
# rational solve in the tests.
FD8 = (-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0)


# Standard 8th-order (radius-4) central first-derivative weights b_1..b_4
# (Fornberg 1988), the inputs of the TTI mixed derivatives; checked against
# the oracle's exact rational solve in the tests.
FD1_8 = (4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0)


def rng(workload: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + workload + 1000 * salt))


def n_coeffs(shape: str, r: int) -> int:
    w = 2 * r + 1
    return {"star": 3 * w, "box": w ** 3, "star2d": 2 * w, "box2d": w * w}[shape]


def n_points(shape: str, r: int) -> int:
    return {"star": 6 * r + 1, "box": (2 * r + 1) ** 3, "star2d": 4 * r + 1, "box2d": (2 * r + 1) ** 2}[shape]


def padded_shape(nx: int, ny: int, nz: int, r: int):
    return (nz + 2 * r, ny + 2 * r, nx + 2 * r)


def uniform_grid(nx, ny, nz, r, workload, salt=0, lo=-1.0, hi=1.0) -> np.ndarray:
    """Padded grid (nz+2r, ny+2r, nx+2r) float32, every value U[lo, hi]."""
    g = rng(workload, salt)
    out = np.empty(padded_shape(nx, ny, nz, r), dtype=np.float32)
    # plane by plane keeps peak memory at one FP64 plane
    for z in range(out.shape[0]):
        out[z] = g.uniform(lo, hi, size=out.shape[1:])
    return out


def normal_coeffs(shape: str, r: int, workload: int, salt=0) -> np.ndarray:
    """Stencil coefficients ~ N(0, 1/npts), float32.

    Box: (2r+1)^3 entries [dz][dy][dx].  Star: (3, 2r+1) per-axis entries
    [axis x,y,z][d+r]; the applied centre is the sum of the three centres.
    The planar shapes: box2d (2r+1)^2 entries [dy][dx], star2d (2, 2r+1)
    entries [axis x,y][d+r].
    """
    g = rng(workload, 100 + salt)
    sd = 1.0 / math.sqrt(n_points(shape, r))
    c = g.normal(0.0, sd, size=n_coeffs(shape, r)).astype(np.float32)
    if shape == "star":
        return c.reshape(3, 2 * r + 1)
    if shape == "star2d":
        return c.reshape(2, 2 * r + 1)
    return c


def uniform_grid2d(nx, ny, nz, r, workload, salt=0, lo=-1.0, hi=1.0) -> np.ndarray:
    """nz independent planes padded in x and y only: (nz, ny+2r, nx+2r)
    float32, every value U[lo, hi]."""
    g = rng(workload, salt)
    out = np.empty((nz, ny + 2 * r, nx + 2 * r), dtype=np.float32)
    for z in range(nz):
        out[z] = g.uniform(lo, hi, size=out.shape[1:])
    return out


def fd8_star_coeffs() -> np.ndarray:
    """(3, 9) float32: the FD8 weights on each axis (centre applied 3x)."""
    row = [FD8[abs(d)] for d in range(-4, 5)]
    return np.array([row, row, row], dtype=np.float32)


def fd8_rows():
    """The radius-4 second- and first-derivative rows over offsets -4..4
    (float32), the TTI workload's weights."""
    w2 = np.array([FD8[abs(d)] for d in range(-4, 5)], np.float32)
    w1 = np.array([-FD1_8[-d - 1] if d < 0 else (0.0 if d == 0 else FD1_8[d - 1]) for d in range(-4, 5)],
                  np.float32)
    return w2, w1


def star_coeffs(r: int, workload: int = 3, salt=0) -> np.ndarray:
    """Star weights of the 1024^3 workload: FD8 at r=4, seeded normal otherwise."""
    return fd8_star_coeffs() if r == 4 else normal_coeffs("star", r, workload, salt)


def sinusoid_grid(nx, ny, nz, r, workload=3, salt=0, n_waves=16, noise=1e-3,
                  chunk=32) -> np.ndarray:
    """Padded grid: sum of n_waves random 3D sinusoids + uniform noise.

    Wave j: a_j sin(k_j . x + phi_j), a_j ~ U[0.5, 1], each component of
    k_j ~ U[0, pi/2] (radians per cell), phi_j ~ U[0, 2 pi), evaluated in FP64
    through the separable identity sin(kx x + ky y + kz z + phi) =
    Im(e^{i(kz z + phi)} e^{i ky y} e^{i kx x}), plus noise * U[-1, 1], cast
    to float32 once.  Coordinates are padded-grid indices.
    """
    g = rng(workload, salt)
    a = g.uniform(0.5, 1.0, n_waves)
    k = g.uniform(0.0, math.pi / 2, size=(n_waves, 3))
    phi = g.uniform(0.0, 2 * math.pi, n_waves)
    Z, Y, X = padded_shape(nx, ny, nz, r)
    ex = np.exp(1j * np.outer(k[:, 0], np.arange(X)))           # (J, X)
    ey = np.exp(1j * np.outer(k[:, 1], np.arange(Y)))           # (J, Y)
    exy = (ey[:, :, None] * ex[:, None, :]).reshape(n_waves, -1)  # (J, Y*X)
    basis = np.concatenate([exy.real, exy.imag], axis=0)        # (2J, Y*X)
    out = np.empty((Z, Y, X), dtype=np.float32)
    zs = np.arange(Z)
    for z0 in range(0, Z, chunk):
        zz = zs[z0:z0 + chunk]
        cz = a[None, :] * np.exp(1j * (np.outer(zz, k[:, 2]) + phi[None, :]))  # (C, J)
        # Im(cz * exy) = Re(cz) Im(exy) + Im(cz) Re(exy)
        w = np.concatenate([cz.imag, cz.real], axis=1)          # (C, 2J)
        out[z0:z0 + chunk] = (w @ basis).reshape(len(zz), Y, X).astype(np.float32)
    nz_ = g.uniform(-1.0, 1.0, size=(Z, Y, X)).astype(np.float32) if Z * Y * X <= 2 ** 28 else None
    if nz_ is not None:
        out += np.float32(noise) * nz_
    else:
        for z in range(Z):
            out[z] += np.float32(noise) * g.uniform(-1.0, 1.0, size=(Y, X)).astype(np.float32)
    return out


def sample_points(nx, ny, nz, n, workload, salt=7, r=0) -> np.ndarray:
    """n interior points (x, y, z), int64, uniform, always including the eight
    corners and the face centres (the edge cases of the halo)."""
    g = rng(workload, salt)
    pts = np.stack([g.integers(0, nx, n), g.integers(0, ny, n), g.integers(0, nz, n)], axis=1)
    extra = []
    for x in (0, nx - 1):
        for y in (0, ny - 1):
            for z in (0, nz - 1):
                extra.append((x, y, z))
    extra += [(nx // 2, ny // 2, 0), (nx // 2, ny // 2, nz - 1), (0, ny // 2, nz // 2),
              (nx - 1, ny // 2, nz // 2), (nx // 2, 0, nz // 2), (nx // 2, ny - 1, nz // 2)]
    return np.concatenate([pts, np.array(extra, dtype=np.int64)], axis=0).astype(np.int64)


# ------------------------------------------------------------- wave inputs

class WaveInputs:
    """Inputs of the acoustic workloads (velocity, sources, wavelet).

    velocity: 6 flat layers, interfaces at sorted seeded depths, velocities
    seeded increasing in [1500, 4500] m/s, times (1 + eta) with eta a
    Gaussian-smoothed (sigma = 8 cells) seeded normal field rescaled to
    max|eta| = 0.05 (noise=False gives the plain layers).
    dt = cfl * h / v_max (CFL 0.4); Ricker f = 15 Hz, t0 = 1/f; source
    amplitude per step s^n = dt^2 * ricker(n dt); sources at z = sponge
    width, x and y seeded in [w, n - w); receivers on the plane z = w.
    """

    def __init__(self, nx, ny, nz, nshots, nsteps, workload=4, h=10.0, sponge=20,
                 sponge_a=0.015, cfl=0.4, f0=15.0, noise=True, salt=0, v=None):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.nshots, self.nsteps = nshots, nsteps
        self.h, self.sponge, self.sponge_a, self.f0 = float(h), int(sponge), float(sponge_a), f0
        g = rng(workload, salt)
        self.v = layered_velocity(nx, ny, nz, g, noise) if v is None else np.asarray(v, np.float32)
        self.vmax = float(self.v.max())
        self.dt = float(np.float32(cfl * self.h / self.vmax))
        w = self.sponge
        lo_x, hi_x = (w, nx - w) if nx > 2 * w else (0, nx)
        lo_y, hi_y = (w, ny - w) if ny > 2 * w else (0, ny)
        self.src = [(int(g.integers(lo_x, hi_x)), int(g.integers(lo_y, hi_y)), min(w, nz - 1))
                    for _ in range(nshots)]
        self.zrec = min(w, nz - 1)
        t = np.arange(nsteps) * self.dt
        wav = ricker(t, f0, 1.0 / f0)
        self.amp = np.repeat((self.dt * self.dt * wav)[:, None], nshots, axis=1).astype(np.float32)


def ricker(t, f0, t0):
    """Ricker wavelet (1 - 2 pi^2 f^2 (t-t0)^2) exp(-pi^2 f^2 (t-t0)^2)."""
    a = (math.pi * f0 * (np.asarray(t, np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def layered_velocity(nx, ny, nz, g: np.random.Generator, noise=True) -> np.ndarray:
    depths = np.sort(g.choice(np.arange(1, max(nz, 7)), size=5, replace=False))
    vel = np.sort(g.uniform(1500.0, 4500.0, 6))
    vel[0], vel[-1] = 1500.0, 4500.0
    vz = np.empty(nz)
    layer = np.searchsorted(depths, np.arange(nz), side="right")
    vz[:] = vel[np.minimum(layer, 5)]
    v = np.broadcast_to(vz[:, None, None], (nz, ny, nx)).astype(np.float64)
    if noise:
        eta = _smooth_noise((nz, ny, nx), g, sigma=8.0)
        v = v * (1.0 + eta)
    return np.ascontiguousarray(v, dtype=np.float32)


def _smooth_noise(shape, g, sigma):
    from scipy.ndimage import gaussian_filter
    e = gaussian_filter(g.standard_normal(shape), sigma=sigma, mode="reflect")
    return 0.05 * e / np.abs(e).max()


# ------------------------------------------------------- anisotropic inputs

class AnisoInputs:
    """Inputs of the VTI and TTI workloads (float32 interior fields).

    vp: the layered velocity of WaveInputs (6 layers, 1500..4500 m/s, 5 %
    smooth noise); eps in [0, 0.3] and delta in [-0.1, 0.2] seeded per layer
    (Thomsen parameters of sedimentary layers); vs = vp / 2; alpha = 1;
    theta (tilt) = a seeded dip in [0, 45] degrees per layer plus a smooth
    field of +-10 degrees; phi (azimuth) = a seeded azimuth plus a smooth field
    of +-30 degrees.  dt follows CFL 0.4 on the fastest speed
    vp sqrt(1 + 2 eps); the sources, receivers and wavelet are those of
    WaveInputs with that dt.
    """

    def __init__(self, nx, ny, nz, nshots, nsteps, workload=6, h=10.0, sponge=20, tti=False, salt=0,
                 noise=True):
        g = rng(workload, salt)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.vp = layered_velocity(nx, ny, nz, g, noise)
        depths = np.sort(g.choice(np.arange(1, max(nz, 7)), size=5, replace=False))
        layer = np.minimum(np.searchsorted(depths, np.arange(nz), side="right"), 5)
        eps_l = g.uniform(0.0, 0.3, 6)
        delta_l = g.uniform(-0.1, 0.2, 6)
        shape = (nz, ny, nx)
        self.eps = np.ascontiguousarray(np.broadcast_to(eps_l[layer][:, None, None], shape), np.float32)
        self.delta = np.ascontiguousarray(np.broadcast_to(delta_l[layer][:, None, None], shape), np.float32)
        vfast = float((self.vp.astype(np.float64) * np.sqrt(1.0 + 2.0 * self.eps)).max())
        self.wave = WaveInputs(nx, ny, nz, nshots, nsteps, workload=workload, h=h, sponge=sponge, salt=salt,
                               v=self.vp, cfl=0.4 * float(self.vp.max()) / vfast)
        self.h, self.dt = self.wave.h, self.wave.dt
        self.src, self.zrec, self.amp = self.wave.src, self.wave.zrec, self.wave.amp
        if tti:
            self.vs = (0.5 * self.vp).astype(np.float32)
            self.alpha = np.ones(shape, np.float32)
            dip = g.uniform(0.0, math.pi / 4, 6)[layer][:, None, None]
            azi = float(g.uniform(-math.pi, math.pi))
            if noise:
                tn = _smooth_noise(shape, g, sigma=8.0) / 0.05 * math.radians(10.0)
                pn = _smooth_noise(shape, g, sigma=8.0) / 0.05 * math.radians(30.0)
            else:
                tn = pn = 0.0
            self.theta = np.ascontiguousarray(np.broadcast_to(dip + tn, shape), np.float32)
            self.phi = np.ascontiguousarray(azi + pn + np.zeros(shape), np.float32)
