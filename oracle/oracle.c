/*
 * oracle.c -- plain, slow, FP64 CPU reference of the stencil sweep and of the
 * acoustic wave step and its adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Everything here is the plain definition written out, one output point at a
 * time, in double precision:
 *
 *   star (paper Sec. 1, Fig. 1; Sec. 4.1): the point is updated from
 *     neighbours along the three coordinate axes only,
 *       out(x,y,z) = sum_{d=-r..r} cx[d] in(x+d,y,z) + cy[d] in(x,y+d,z)
 *                                 + cz[d] in(x,y,z+d)
 *     so the applied centre weight is cx[0]+cy[0]+cz[0];
 *   box  (paper Sec. 1, Fig. 1): every point of the (2r+1)^3 cube,
 *       out(x,y,z) = sum_{dz,dy,dx} c[dz][dy][dx] in(x+dx,y+dy,z+dz).
 *
 * The paper's banded-matrix decomposition (Sec. 4.1) and its box
 * decomposition (Sec. 4.3, "redundant-access zeroing") reach exactly this
 * result up to summation order; the oracle uses neither.
 *
 * Layouts.  The input grid is padded by the radius r on every face; element
 * (X,Y,Z) of the padded grid (0 <= X < nx+2r, ...) lives at
 * Z*pz + Y*py + X (pitches in elements).  Output point (x,y,z) of the
 * nx*ny*nz interior reads padded element (x+r, y+r, z+r) as its centre and is
 * stored densely at (z*ny + y)*nx + x.
 *
 * The wave step and its adjoint follow the discretisation stated in the
 * functions below; the paper names reverse time migration (Sec. 2.1,
 * Sec. 5.6) but prints no discretisation, so the readings are those listed in
 * the design notes (leapfrog, Cerjan sponge, zero halo).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(X, Y, Z, py, pz) ((int64_t)(Z) * (pz) + (int64_t)(Y) * (py) + (int64_t)(X))

/* ---------------------------------------------------------------- sweeps */

/* One star output point.  c has 3*(2r+1) entries: [axis x,y,z][d+r]. */
static double star_point(int r, const double *c, const double *in, int64_t py,
                         int64_t pz, int64_t x, int64_t y, int64_t z)
{
    const int w = 2 * r + 1;
    const int64_t X = x + r, Y = y + r, Z = z + r;
    double acc = 0.0;
    for (int d = -r; d <= r; ++d) {
        acc += c[0 * w + d + r] * in[IDX(X + d, Y, Z, py, pz)];
        acc += c[1 * w + d + r] * in[IDX(X, Y + d, Z, py, pz)];
        acc += c[2 * w + d + r] * in[IDX(X, Y, Z + d, py, pz)];
    }
    return acc;
}

/* One box output point.  c has (2r+1)^3 entries: [dz+r][dy+r][dx+r]. */
static double box_point(int r, const double *c, const double *in, int64_t py,
                        int64_t pz, int64_t x, int64_t y, int64_t z)
{
    const int w = 2 * r + 1;
    const int64_t X = x + r, Y = y + r, Z = z + r;
    double acc = 0.0;
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx)
                acc += c[((dz + r) * w + (dy + r)) * w + (dx + r)] *
                       in[IDX(X + dx, Y + dy, Z + dz, py, pz)];
    return acc;
}

/* Full sweep over the interior; shape 0 = star, 1 = box. */
void orc_stencil(int shape, int r, const double *c, const double *in, int64_t py,
                 int64_t pz, int64_t nx, int64_t ny, int64_t nz, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x)
                out[(z * ny + y) * nx + x] =
                    shape == 0 ? star_point(r, c, in, py, pz, x, y, z)
                               : box_point(r, c, in, py, pz, x, y, z);
}

/* Sampled points: xyz holds npts triples (x,y,z) of interior coordinates. */
void orc_stencil_points(int shape, int r, const double *c, const double *in,
                        int64_t py, int64_t pz, int64_t npts, const int64_t *xyz,
                        double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npts; ++i) {
        const int64_t x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        out[i] = shape == 0 ? star_point(r, c, in, py, pz, x, y, z)
                            : box_point(r, c, in, py, pz, x, y, z);
    }
}

/* Same as orc_stencil_points but reading an FP32 grid (each value promoted to
 * double before use), so the full-size inputs need no FP64 copy. */
void orc_stencil_points_f32(int shape, int r, const double *c, const float *in,
                            int64_t py, int64_t pz, int64_t npts,
                            const int64_t *xyz, double *out)
{
    const int w = 2 * r + 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npts; ++i) {
        const int64_t X = xyz[3 * i] + r, Y = xyz[3 * i + 1] + r, Z = xyz[3 * i + 2] + r;
        double acc = 0.0;
        if (shape == 0) {
            for (int d = -r; d <= r; ++d) {
                acc += c[0 * w + d + r] * (double)in[IDX(X + d, Y, Z, py, pz)];
                acc += c[1 * w + d + r] * (double)in[IDX(X, Y + d, Z, py, pz)];
                acc += c[2 * w + d + r] * (double)in[IDX(X, Y, Z + d, py, pz)];
            }
        } else {
            for (int dz = -r; dz <= r; ++dz)
                for (int dy = -r; dy <= r; ++dy)
                    for (int dx = -r; dx <= r; ++dx)
                        acc += c[((dz + r) * w + (dy + r)) * w + (dx + r)] *
                               (double)in[IDX(X + dx, Y + dy, Z + dz, py, pz)];
        }
        out[i] = acc;
    }
}

/* ------------------------------------------------------- acoustic wave */

/*
 * Cerjan et al. (1985) absorbing sponge, one axis: for the cell at 0-based
 * index i of n, d = min(i, n-1-i) is its distance to the nearest face and
 *   g(i) = exp(-(a*(w-d))^2)  if d < w,   g(i) = 1 otherwise.
 * The 3D factor is g(x)*g(y)*g(z).
 */
void orc_sponge_1d(int64_t n, int w, double a, double *g)
{
    for (int64_t i = 0; i < n; ++i) {
        const int64_t d = i < n - 1 - i ? i : n - 1 - i;
        if (d < w) {
            const double t = a * (double)(w - d);
            g[i] = exp(-t * t);
        } else {
            g[i] = 1.0;
        }
    }
}

/*
 * One leapfrog step of the damped acoustic wave equation, one shot:
 *   a_next = G * ( (2 + m*L) a_cur - G * a_prev + s )
 * on the interior, with L the star stencil of radius r (coefficients c,
 * [axis][d+r], unscaled; 1/h^2 lives in m = v^2 dt^2 / h^2), G = gx*gy*gz and
 * s = s_amp at the source point (sx,sy,sz) only (sx < 0: no source).
 * All fields are padded by r with a zero halo and share pitches py, pz; m is
 * padded too (its halo is never read here).  The halo of a_next is not
 * written.
 */
void orc_wave_step(int r, const double *c, int64_t nx, int64_t ny, int64_t nz,
                   int64_t py, int64_t pz, const double *m, const double *gx,
                   const double *gy, const double *gz, const double *a_cur,
                   const double *a_prev, double *a_next, int64_t sx, int64_t sy,
                   int64_t sz, double s_amp)
{
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t p = IDX(x + r, y + r, z + r, py, pz);
                const double g = gx[x] * gy[y] * gz[z];
                const double lap = star_point(r, c, a_cur, py, pz, x, y, z);
                double v = 2.0 * a_cur[p] + m[p] * lap - g * a_prev[p];
                if (x == sx && y == sy && z == sz)
                    v += s_amp;
                a_next[p] = g * v;
            }
}

/*
 * One step of the discrete adjoint of orc_wave_step (discretise, then
 * differentiate).  Writing the forward step as
 *   a^{n+1} = G(2 + M L) a^n - G^2 a^{n-1} + G s^n,    d^n = R a^n,
 * with M = diag(m), G = diag(g), R the restriction to the receiver plane
 * z = zrec, the adjoint state of J = 1/2 sum_n |d^n - d_obs^n|^2 obeys
 *   lam^n = R^T r^n + (2 + L M) G lam^{n+1} - G^2 lam^{n+2}
 * (L is symmetric for symmetric weights and a zero halo), and
 *   dJ/dm += G lam^{n+1} * (L a^n).
 * lam1 = lam^{n+1}, lam2 = lam^{n+2}, resid = r^n (ny*nx, may be NULL),
 * a_n = forward state a^n (may be NULL: no gradient term), lam0 = output
 * lam^n (interior written, halo untouched), grad = nx*ny*nz dense, accumulated.
 * q is caller-provided padded scratch with a zero halo (same pitches).
 */
void orc_wave_adjoint_step(int r, const double *c, int64_t nx, int64_t ny,
                           int64_t nz, int64_t py, int64_t pz, const double *m,
                           const double *gx, const double *gy, const double *gz,
                           const double *lam1, const double *lam2,
                           const double *resid, int64_t zrec, const double *a_n,
                           double *lam0, double *grad, double *q)
{
    /* q = m * g * lam^{n+1} on the interior; its halo stays zero. */
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t p = IDX(x + r, y + r, z + r, py, pz);
                q[p] = m[p] * gx[x] * gy[y] * gz[z] * lam1[p];
            }
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t p = IDX(x + r, y + r, z + r, py, pz);
                const double g = gx[x] * gy[y] * gz[z];
                double v = 2.0 * g * lam1[p] + star_point(r, c, q, py, pz, x, y, z) -
                           g * g * lam2[p];
                if (resid && z == zrec)
                    v += resid[y * nx + x];
                lam0[p] = v;
                if (a_n)
                    grad[(z * ny + y) * nx + x] +=
                        g * lam1[p] * star_point(r, c, a_n, py, pz, x, y, z);
            }
}

/* <u, w> over the interior of two padded fields (for energy and dot tests). */
double orc_dot_interior(int r, int64_t nx, int64_t ny, int64_t nz, int64_t py,
                        int64_t pz, const double *u, const double *w)
{
    double s = 0.0;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t p = IDX(x + r, y + r, z + r, py, pz);
                s += u[p] * w[p];
            }
    return s;
}

/* Thread count of the parallel loops above (n > 0 sets it for the calling
 * thread's later loops; n = 0 leaves it); returns the count before the call.
 * Lets a caller time the oracle on one core as well as on all of them. */
int orc_set_threads(int n)
{
    const int old = omp_get_max_threads();
    if (n > 0) omp_set_num_threads(n);
    return old;
}
