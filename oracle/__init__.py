"""FP64 CPU oracle of the stencil sweep, the wave step and its adjoint.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_2507_11067_gb300``) and never imports it;
the two meet only through the seeded inputs of ``workloads``.

What it computes, and where the paper defines it:

* ``stencil`` / ``stencil_points``: the star and box sweeps of Sec. 1
  (Fig. 1) -- the plain definition, one point at a time, in FP64
  (``oracle.c``).  The banded-matrix form of Sec. 4.1 reaches the same
  values up to summation order.
* ``fd2_weights``: the central second-derivative weights of radius r used for
  high-order finite differences (Sec. 2.1: radius 4 gives 8th-order accuracy),
  obtained by solving the moment (Taylor) conditions in exact rationals.
* ``wave_forward`` / ``wave_gradient``: the acoustic wave step used in place
  of the paper's RTM kernels (Sec. 2.1, Sec. 5.6) and its discrete adjoint;
  the paper prints no discretisation, so the step is the leapfrog form
  written in ``oracle.c``.

Parity pins (tests/test_oracle_*.py) tie every function here to facts that do
not depend on this code: closed-form weights, polynomial exactness, the
Fourier symbol, scipy.ndimage.correlate, brute force on 8^3 grids,
adjointness, energy conservation, time reversibility and finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain C, OpenMP) into oracle/_build."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
    P = ctypes.c_void_p
    lib.orc_stencil.argtypes = [i32, i32, P, P, i64, i64, i64, i64, i64, P]
    lib.orc_stencil_points.argtypes = [i32, i32, P, P, i64, i64, i64, P, P]
    lib.orc_stencil_points_f32.argtypes = [i32, i32, P, P, i64, i64, i64, P, P]
    lib.orc_sponge_1d.argtypes = [i64, i32, d, P]
    lib.orc_wave_step.argtypes = [i32, P, i64, i64, i64, i64, i64, P, P, P, P, P, P, P,
                                  i64, i64, i64, d]
    lib.orc_wave_adjoint_step.argtypes = [i32, P, i64, i64, i64, i64, i64, P, P, P, P, P,
                                          P, P, i64, P, P, P, P]
    lib.orc_dot_interior.argtypes = [i32, i64, i64, i64, i64, i64, P, P]
    lib.orc_dot_interior.restype = d
    lib.orc_set_threads.argtypes = [i32]
    lib.orc_set_threads.restype = i32
    _lib = lib
    return lib


def set_threads(n: int) -> int:
    """Threads of oracle.c's parallel loops from now on in the calling thread
    (n = 0 leaves the count); returns the count before the call."""
    return int(_load().orc_set_threads(int(n)))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


SHAPES = {"star": 0, "box": 1}


def n_coeffs(shape: str, r: int) -> int:
    """Number of stored coefficients: 3(2r+1) per-axis weights for a star,
    (2r+1)^3 for a box (Sec. 1, Fig. 1; Table I point counts); the planar
    star2d and box2d of Table I's 2D kernels: 2(2r+1) and (2r+1)^2."""
    w = 2 * r + 1
    return {"star": 3 * w, "box": w ** 3, "star2d": 2 * w, "box2d": w * w}[shape]


def n_points(shape: str, r: int) -> int:
    """Distinct stencil points: 6r+1 for a 3D star, (2r+1)^3 for a 3D box,
    4r+1 and (2r+1)^2 for their planar counterparts."""
    return {"star": 6 * r + 1, "box": (2 * r + 1) ** 3, "star2d": 4 * r + 1, "box2d": (2 * r + 1) ** 2}[shape]


# ------------------------------------------------------------------ sweeps

def _check_grid(shape, r, coeffs, grid):
    if r < 1:
        raise ValueError("radius must be >= 1")
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64).reshape(-1))
    if c.size != n_coeffs(shape, r):
        raise ValueError(f"{shape} r={r} needs {n_coeffs(shape, r)} coefficients, got {c.size}")
    g = np.asarray(grid)
    if g.ndim != 3:
        raise ValueError("padded grid must be 3D (z, y, x)")
    nz, ny, nx = (s - 2 * r for s in g.shape)
    if min(nx, ny, nz) < 0:
        raise ValueError("grid smaller than its halo")
    return c, nx, ny, nz


def stencil(shape: str, r: int, coeffs, grid) -> np.ndarray:
    """Apply the star or box stencil to a padded grid (z, y, x), FP64 result.

    ``grid`` has shape (nz+2r, ny+2r, nx+2r); the result is (nz, ny, nx).
    FP32 inputs are promoted exactly to FP64 (Sec. 1 definition; oracle.c).
    """
    c, nx, ny, nz = _check_grid(shape, r, coeffs, grid)
    g = np.ascontiguousarray(grid, dtype=np.float64)
    out = np.empty((nz, ny, nx), dtype=np.float64)
    if out.size:
        _load().orc_stencil(SHAPES[shape], r, _ptr(c), _ptr(g), g.shape[2],
                            g.shape[1] * g.shape[2], nx, ny, nz, _ptr(out))
    return out


def stencil2d(shape: str, r: int, coeffs, grid) -> np.ndarray:
    """The planar stencils of Table I's 2D kernels on nz independent planes.

    ``grid`` is (nz, ny+2r, nx+2r), padded in x and y only; the FP64 result
    (nz, ny, nx) is, for box2d with weights c[dy][dx],
        out(x, y, z) = sum_{dy,dx} c[dy][dx] in(x+r+dx, y+r+dy, z),
    and for star2d with per-axis weights cx, cy the x line plus the y line
    (the applied centre is cx[0] + cy[0]) -- Sec. 1, Fig. 1 in one plane.
    """
    if shape not in ("star2d", "box2d") or r < 1:
        raise ValueError("planar shape star2d or box2d, radius >= 1")
    c = np.asarray(coeffs, dtype=np.float64).reshape(-1)
    if c.size != n_coeffs(shape, r):
        raise ValueError(f"{shape} r={r} needs {n_coeffs(shape, r)} coefficients, got {c.size}")
    g = np.asarray(grid, dtype=np.float64)
    if g.ndim != 3:
        raise ValueError("grid must be (nz, ny+2r, nx+2r)")
    nz, ny, nx = g.shape[0], g.shape[1] - 2 * r, g.shape[2] - 2 * r
    if min(nx, ny) < 0:
        raise ValueError("grid smaller than its halo")
    w = 2 * r + 1
    out = np.zeros((nz, ny, nx))
    if shape == "box2d":
        c = c.reshape(w, w)
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                out += c[dy + r, dx + r] * g[:, r + dy:r + dy + ny, r + dx:r + dx + nx]
    else:
        cx, cy = c[:w], c[w:]
        for d in range(-r, r + 1):
            out += cx[d + r] * g[:, r:r + ny, r + d:r + d + nx]
            out += cy[d + r] * g[:, r + d:r + d + ny, r:r + nx]
    return out


def stencil2d_points(shape: str, r: int, coeffs, grid, xyz) -> np.ndarray:
    """stencil2d at the points ``xyz`` (npts, 3) = (x, y, plane) only; the
    grid is read in place."""
    pts = np.asarray(xyz, dtype=np.int64).reshape(-1, 3)
    g = np.asarray(grid)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    c = np.asarray(coeffs, dtype=np.float64).reshape(-1)
    w = 2 * r + 1
    out = np.zeros(len(pts))
    if shape == "box2d":
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                out += c[(dy + r) * w + dx + r] * g[z, y + r + dy, x + r + dx].astype(np.float64)
    elif shape == "star2d":
        for d in range(-r, r + 1):
            out += c[d + r] * g[z, y + r, x + r + d].astype(np.float64)
            out += c[w + d + r] * g[z, y + r + d, x + r].astype(np.float64)
    else:
        raise ValueError("planar shape star2d or box2d")
    return out


def stencil_points(shape: str, r: int, coeffs, grid, xyz) -> np.ndarray:
    """The stencil evaluated only at interior points ``xyz`` (npts, 3) = (x, y, z).

    A float32 grid is read in place (each value promoted to FP64 when used),
    so full-size grids need no FP64 copy.
    """
    c, nx, ny, nz = _check_grid(shape, r, coeffs, grid)
    pts = np.ascontiguousarray(np.asarray(xyz, dtype=np.int64).reshape(-1, 3))
    if pts.size and ((pts < 0).any() or (pts[:, 0] >= nx).any() or (pts[:, 1] >= ny).any()
                     or (pts[:, 2] >= nz).any()):
        raise ValueError("sample point outside the interior")
    out = np.empty(len(pts), dtype=np.float64)
    if not len(pts):
        return out
    g = np.asarray(grid)
    if g.dtype == np.float32 and g.flags.c_contiguous:
        _load().orc_stencil_points_f32(SHAPES[shape], r, _ptr(c), _ptr(g), g.shape[2],
                                       g.shape[1] * g.shape[2], len(pts), _ptr(pts), _ptr(out))
    else:
        g = np.ascontiguousarray(g, dtype=np.float64)
        _load().orc_stencil_points(SHAPES[shape], r, _ptr(c), _ptr(g), g.shape[2],
                                   g.shape[1] * g.shape[2], len(pts), _ptr(pts), _ptr(out))
    return out


# ------------------------------------------------------- FD weights (exact)

def fd2_weights(r: int) -> list:
    """Central 2nd-derivative weights c_0..c_r of radius r, exact rationals.

    The symmetric stencil sum_k c_|k| f(k) must reproduce d^2/dx^2 on the
    monomials x^0, x^2, ..., x^{2r} at x = 0 (odd moments vanish by symmetry):
        c_0 + 2 sum_k c_k      = 0
        2 sum_k c_k k^{2j}     = 2 delta_{j,1}      (j = 1..r)
    Solved by Gauss-Jordan elimination over Fractions.  Radius 4 gives the
    8th-order weights that Sec. 2.1 associates with RTM.
    """
    n = r + 1
    A = [[Fraction(0)] * n for _ in range(n)]
    b = [Fraction(0)] * n
    A[0][0] = Fraction(1)
    for k in range(1, n):
        A[0][k] = Fraction(2)
    for j in range(1, n):
        for k in range(1, n):
            A[j][k] = Fraction(2 * k ** (2 * j))
        b[j] = Fraction(2) if j == 1 else Fraction(0)
    # Gauss-Jordan
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
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


def fd2_star_coeffs(r: int) -> np.ndarray:
    """Per-axis star coefficients (3, 2r+1) from fd2_weights, as FP64.

    Each axis carries the full 1D weight set, so the applied centre is the
    sum of the three axis centres (3 c_0)."""
    w = fd2_weights(r)
    row = [float(w[abs(d)]) for d in range(-r, r + 1)]
    return np.array([row, row, row], dtype=np.float64)


# ------------------------------------------------------------ wave (FP64)

def sponge_1d(n: int, width: int, a: float) -> np.ndarray:
    """Cerjan sponge profile along one axis (see orc_sponge_1d)."""
    g = np.empty(n, dtype=np.float64)
    if n:
        _load().orc_sponge_1d(n, width, float(a), _ptr(g))
    return g


def model_m(v, dt: float, h: float) -> np.ndarray:
    """m = v^2 dt^2 / h^2, the coefficient of L in the leapfrog step."""
    v = np.asarray(v, dtype=np.float64)
    return v * v * (dt * dt) / (h * h)


def pad(field, r: int) -> np.ndarray:
    """Interior (nz, ny, nx) -> padded FP64 with a zero halo of width r."""
    f = np.asarray(field, dtype=np.float64)
    out = np.zeros(tuple(s + 2 * r for s in f.shape), dtype=np.float64)
    out[r:-r, r:-r, r:-r] = f
    return out


class WaveProblem:
    """Geometry and coefficients of the damped acoustic wave step (FP64).

    coeffs: star (3, 2r+1) unscaled weights; m_int: (nz, ny, nx) interior
    m = v^2 dt^2/h^2; sponge: (width, a) or None (no damping, G = 1);
    src: list of (x, y, z) per shot; amp: (nsteps, nshots) source values s^n;
    zrec: receiver plane (interior z index).
    """

    def __init__(self, r, coeffs, m_int, sponge, src, amp, zrec):
        self.r = int(r)
        self.c = np.ascontiguousarray(np.asarray(coeffs, np.float64).reshape(-1))
        if self.c.size != n_coeffs("star", self.r):
            raise ValueError("wave step needs star coefficients")
        self.nz, self.ny, self.nx = np.asarray(m_int).shape
        self.m = pad(m_int, self.r)
        if sponge is None:
            self.gx, self.gy, self.gz = (np.ones(n) for n in (self.nx, self.ny, self.nz))
        else:
            wdt, a = sponge
            self.gx, self.gy, self.gz = (sponge_1d(n, wdt, a) for n in (self.nx, self.ny, self.nz))
        self.src = [tuple(int(v) for v in s) for s in src]
        self.amp = np.asarray(amp, dtype=np.float64)
        self.zrec = int(zrec)
        P = self.m.shape
        self.py, self.pz = P[2], P[1] * P[2]

    def zeros(self):
        return np.zeros_like(self.m)

    def step(self, a_cur, a_prev, shot: int, n: int):
        """a^{n+1} from a^n, a^{n-1} for one shot (oracle.c orc_wave_step)."""
        out = self.zeros()
        sx, sy, sz = self.src[shot] if self.src else (-1, -1, -1)
        s = float(self.amp[n, shot]) if self.amp.size else 0.0
        _load().orc_wave_step(self.r, _ptr(self.c), self.nx, self.ny, self.nz, self.py,
                              self.pz, _ptr(self.m), _ptr(self.gx), _ptr(self.gy),
                              _ptr(self.gz), _ptr(a_cur), _ptr(a_prev), _ptr(out),
                              sx, sy, sz, s)
        return out

    def laplacian(self, a):
        """L a on the interior (nz, ny, nx), unscaled star."""
        return stencil("star", self.r, self.c.reshape(3, -1), a)

    def record(self, a):
        r = self.r
        return a[r + self.zrec, r:r + self.ny, r:r + self.nx].copy()

    def forward(self, nsteps: int, keep_states: bool = False):
        """Run nsteps leapfrog steps from a^0 = a^{-1} = 0 for every shot.

        Returns records d[n-1, shot] = R a^n for n = 1..nsteps and, when asked,
        the states a^0..a^nsteps per shot.
        """
        nshots = len(self.src)
        rec = np.zeros((nsteps, nshots, self.ny, self.nx))
        states = [[self.zeros()] for _ in range(nshots)] if keep_states else None
        for s in range(nshots):
            prev, cur = self.zeros(), self.zeros()
            for n in range(nsteps):
                nxt = self.step(cur, prev, s, n)
                prev, cur = cur, nxt
                rec[n, s] = self.record(cur)
                if keep_states:
                    states[s].append(cur)
        return rec, states

    def adjoint_step(self, lam1, lam2, resid, a_n, grad):
        """lam^n from lam^{n+1}, lam^{n+2}; grad += g lam^{n+1} (L a^n)."""
        out = self.zeros()
        q = self.zeros()
        rp = None if resid is None else np.ascontiguousarray(resid, dtype=np.float64)
        _load().orc_wave_adjoint_step(
            self.r, _ptr(self.c), self.nx, self.ny, self.nz, self.py, self.pz,
            _ptr(self.m), _ptr(self.gx), _ptr(self.gy), _ptr(self.gz), _ptr(lam1),
            _ptr(lam2), None if rp is None else _ptr(rp), self.zrec,
            None if a_n is None else _ptr(a_n), _ptr(out), _ptr(grad), _ptr(q))
        return out

    def gradient_m(self, resid, states):
        """dJ/dm for J = 1/2 sum_n |d^n - d_obs^n|^2 given resid[n-1, shot] =
        d^n - d_obs^n and the forward states a^0..a^Nt of every shot."""
        nsteps = resid.shape[0]
        grad = np.zeros((self.nz, self.ny, self.nx))
        for s in range(resid.shape[1]):
            lam1, lam2 = self.zeros(), self.zeros()          # lam^{Nt+1}, lam^{Nt+2}
            for n in range(nsteps, 0, -1):                     # lam^n, n = Nt..1
                lam0 = self.adjoint_step(lam1, lam2, resid[n - 1, s], states[s][n], grad)
                lam2, lam1 = lam1, lam0
            # n = 0 term: g lam^1 (L a^0) with a^0 = 0 contributes nothing
        return grad

    def dot(self, u, w):
        return _load().orc_dot_interior(self.r, self.nx, self.ny, self.nz, self.py, self.pz,
                                        _ptr(np.ascontiguousarray(u)), _ptr(np.ascontiguousarray(w)))


def wave_step_points(r: int, coeffs, m_int, sponge, src, s_amp: float, a_cur, a_prev, xyz) -> np.ndarray:
    """a^{n+1} of one shot at interior points ``xyz`` (npts, 3) = (x, y, z):

        a^{n+1} = G ( 2 a^n + m L a^n - G a^{n-1} + s^n [p = src] ),

    G = g(x) g(y) g(z) the Cerjan profile, L the unscaled star of radius r
    (the damped leapfrog step of WaveProblem.step, written out point by
    point).  a_cur, a_prev: padded fields of the shot (zero halo), read in
    place; m_int: interior m = v^2 dt^2 / h^2; sponge: (width, a) or None;
    src: (x, y, z) of the shot's source; s_amp: its value s^n.
    """
    pts = np.ascontiguousarray(np.asarray(xyz, dtype=np.int64).reshape(-1, 3))
    lap = stencil_points("star", r, np.asarray(coeffs).reshape(3, -1), a_cur, pts)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    nz, ny, nx = np.asarray(m_int).shape
    if sponge is None:
        g = np.ones(len(pts))
    else:
        g = sponge_1d(nx, *sponge)[x] * sponge_1d(ny, *sponge)[y] * sponge_1d(nz, *sponge)[z]
    m = np.asarray(m_int)[z, y, x].astype(np.float64)
    ac = np.asarray(a_cur)[z + r, y + r, x + r].astype(np.float64)
    ap = np.asarray(a_prev)[z + r, y + r, x + r].astype(np.float64)
    s = np.where((x == src[0]) & (y == src[1]) & (z == src[2]), float(s_amp), 0.0)
    return g * (2.0 * ac + m * lap - g * ap + s)


def objective(rec, obs) -> float:
    """J = 1/2 sum |d - d_obs|^2 (FP64)."""
    d = np.asarray(rec, np.float64) - np.asarray(obs, np.float64)
    return 0.5 * float(np.sum(d * d))
