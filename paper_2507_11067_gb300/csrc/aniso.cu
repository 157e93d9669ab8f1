// aniso.cu -- wave steps of the coupled anisotropic systems of the paper's
// Sec. 2.1: VTI (two stresses sigma_H, sigma_V; one fused kernel) and TTI
// (fields p, q with the tilted operators H1, H2; a derivative pass for p,
// then one for q with the coupling and the update fused in).
//
// VTI.  With mh = m (1+2 eps), mv = m sqrt(1+2 delta) (m = vp^2 dt^2/h^2)
// the printed system is
//     sigma_H'' = mh Lh sigma_H + mv Lz sigma_V
//     sigma_V'' = mv Lh sigma_V + mh Lz sigma_H
// (Lh = d_xx + d_yy, Lz = d_zz, unscaled weights).  The library stores the
// medium as mv and rho = mh / mv = (1+2 eps)/sqrt(1+2 delta), so that
//     sigma_H'' = mv      [ rho Lh sigma_H   + Lz sigma_V ]
//     sigma_V'' = mv rho  [ Lh sigma_V / rho + Lz sigma_H ]
// and each field needs ONE register queue of partial sums along z, as the
// acoustic step does: the in-plane part enters the queue at the plane it
// centres, scaled by that plane's rho (or 1/rho), the z part from every
// plane in reach; the output multiplies by mv (mv rho) when it completes.
// One step moves 32 bytes per point: read sigma_H, sigma_V at n and n-1,
// mv and rho; write sigma_H, sigma_V at n+1 (halos served from L2).
#include "common.cuh"
#include "tile.cuh"
#include "wave.cuh"

namespace mms {

namespace {

// Stage s of the ring: [sigma_H plane + halo | sigma_V plane + halo |
// rho tile of the plane itself (its in-plane part) | mv, rho, sigma_H^{n-1},
// sigma_V^{n-1}, sigma_H^n, sigma_V^n tiles of the output plane that the
// plane completes].  Every sub-buffer starts on 128 bytes.
template <int R, int TX, int TY, int S>
struct VtiGeom {
    using G = Geom<R, TX, TY, 1, S>;
    using I = Interior<R, TX>;
    static constexpr int PL = (G::PLANE + 31) & ~31;
    static constexpr int MT = (I::BXI * TY + 31) & ~31;
    static constexpr int OFF_V = PL;
    static constexpr int OFF_RC = 2 * PL;
    static constexpr int OFF_MV = OFF_RC + MT;
    static constexpr int OFF_RZ = OFF_MV + MT;
    static constexpr int OFF_HP = OFF_RZ + MT;
    static constexpr int OFF_VP = OFF_HP + MT;
    static constexpr int OFF_HC = OFF_VP + MT;
    static constexpr int OFF_VC = OFF_HC + MT;
    static constexpr int STAGE = OFF_VC + MT;
    static constexpr size_t SMEM = 128 + (size_t)S * STAGE * 4 + S * sizeof(uint64_t) + 16;
    static_assert(SMEM <= 227 * 1024, "stage ring exceeds shared memory");
};

struct VtiMaps {
    CUtensorMap h, v;                 // sigma^n planes with halo (per shot)
    CUtensorMap rho, mv;              // interior tiles of the medium
    CUtensorMap hp, vp, hc, vc;       // interior tiles of sigma^{n-1}, sigma^n (per shot)
};

template <int R, int TX, int TY, int S>
__global__ void __launch_bounds__(Geom<R, TX, TY, 1, S>::NT)
    vti_fwd_kernel(const __grid_constant__ VtiMaps tm, const __grid_constant__ StarCoef cf,
                   const __grid_constant__ WaveGeo geo, float *__restrict__ hnext, float *__restrict__ vnext,
                   const float *__restrict__ amp, float *__restrict__ rec, int tz, int nzc, int vec,
                   unsigned *err)
{
    using G = Geom<R, TX, TY, 1, S>;
    using V = VtiGeom<R, TX, TY, S>;
    using I = Interior<R, TX>;
    constexpr int W = G::W;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_align128(smem_raw);
    float *stages = reinterpret_cast<float *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)S * V::STAGE * sizeof(float));
    int &abort_flag = *reinterpret_cast<int *>(full + S);

    const int tid = threadIdx.x;
    const int tx = tid % G::NTX, ty = tid / G::NTX;
    const int sh = blockIdx.z / nzc, zc = blockIdx.z % nzc;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, zb = zc * tz;
    const int nzt = min(tz, geo.nz - zb);
    const int P = nzt + 2 * R;
    const int gx = x0 + 4 * tx;
    const int sx = geo.src[sh][0], sy = geo.src[sh][1], sz = geo.src[sh][2];

    auto issue = [&](int j, int s) {
        float *st = stages + (size_t)s * V::STAGE;
        const bool centre = j >= R && j < R + nzt;  // an output plane of this chunk
        const bool done = j >= 2 * R;               // completes output plane j - 2R
        const uint32_t bytes = (2 * G::PLANE + (centre ? I::BXI * TY : 0) + (done ? 6 * I::BXI * TY : 0)) * 4;
        ptx::mbar_arrive_expect_tx(&full[s], bytes);
        ptx::tma_load_4d(st, &tm.h, x0, y0, zb + j, sh, &full[s]);
        ptx::tma_load_4d(st + V::OFF_V, &tm.v, x0, y0, zb + j, sh, &full[s]);
        const int xs = x0 + (R & ~3);
        if (centre) ptx::tma_load_3d(st + V::OFF_RC, &tm.rho, xs, y0 + R, zb + j, &full[s]);
        if (done) {
            const int zp = zb + j - R;  // padded plane of output zo = j - 2R
            ptx::tma_load_3d(st + V::OFF_MV, &tm.mv, xs, y0 + R, zp, &full[s]);
            ptx::tma_load_3d(st + V::OFF_RZ, &tm.rho, xs, y0 + R, zp, &full[s]);
            ptx::tma_load_4d(st + V::OFF_HP, &tm.hp, xs, y0 + R, zp, sh, &full[s]);
            ptx::tma_load_4d(st + V::OFF_VP, &tm.vp, xs, y0 + R, zp, sh, &full[s]);
            ptx::tma_load_4d(st + V::OFF_HC, &tm.hc, xs, y0 + R, zp, sh, &full[s]);
            ptx::tma_load_4d(st + V::OFF_VC, &tm.vc, xs, y0 + R, zp, sh, &full[s]);
        }
    };
    if (tid == 0) {
        ptx::prefetch_tmap(&tm.h);
        ptx::prefetch_tmap(&tm.v);
        ptx::prefetch_tmap(&tm.rho);
        ptx::prefetch_tmap(&tm.mv);
        ptx::prefetch_tmap(&tm.hp);
        ptx::prefetch_tmap(&tm.vp);
#pragma unroll
        for (int s = 0; s < S; ++s) ptx::mbar_init(&full[s], 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();
    if (tid == 0)
        for (int j = 0; j < S && j < P; ++j) issue(j, j);

    float gxs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) gxs[k] = sponge(gx + k, geo.nx, geo.sponge_w, geo.sponge_a);
    const float gys = sponge(y0 + ty, geo.ny, geo.sponge_w, geo.sponge_a);

    // qh: rho Lh sigma_H + Lz sigma_V; qv: Lh sigma_V / rho + Lz sigma_H
    float qh[W][4], qv[W][4];
#pragma unroll
    for (int kk = 0; kk < W; ++kk)
#pragma unroll
        for (int k = 0; k < 4; ++k) qh[kk][k] = qv[kk][k] = 0.f;

    const float samp = amp[sh];
    const int64_t shot_off = (int64_t)sh * geo.ss;
    for (int j = 0; j < P; ++j) {
        const int s = j % S;
        const float *st = stages + (size_t)s * V::STAGE;
        const int zo = j - 2 * R;
        const bool centre = j >= R && j < R + nzt;
        float mv[4], rz[4], hp[4], vp[4], hc[4], vc[4];
        if (ptx::mbar_wait_bounded(&full[s], (uint32_t)(j / S) & 1u, err)) {
            const float *ph = st, *pv = st + V::OFF_V;
            float ch[4], cv[4];
            load_center<R>(ph + (ty + R) * G::BX + 4 * tx, ch);
            load_center<R>(pv + (ty + R) * G::BX + 4 * tx, cv);
            // z part: this plane is offset R - kk from the output plane of slot kk
#pragma unroll
            for (int kk = 0; kk < W; ++kk)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float wz = cf.c[2 * W + 2 * R - kk];
                    qh[kk][k] = fmaf(wz, cv[k], qh[kk][k]);
                    qv[kk][k] = fmaf(wz, ch[k], qv[kk][k]);
                }
            if (centre) {
                float rc[4];
                load_center<I::OFF>(st + V::OFF_RC + ty * I::BXI + 4 * tx, rc);
                float wh[4 * G::NV], wv[4 * G::NV];
                load_row<G::NV>(ph + (ty + R) * G::BX + 4 * tx, wh);
                load_row<G::NV>(pv + (ty + R) * G::BX + 4 * tx, wv);
                float lh[4], lv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    lh[k] = 0.f;
                    lv[k] = 0.f;
#pragma unroll
                    for (int d = -R; d <= R; ++d) {
                        lh[k] = fmaf(cf.c[d + R], wh[k + R + d], lh[k]);
                        lv[k] = fmaf(cf.c[d + R], wv[k + R + d], lv[k]);
                    }
                }
#pragma unroll
                for (int d = -R; d <= R; ++d) {
                    float ah[4], av[4];
                    load_center<R>(ph + (ty + R + d) * G::BX + 4 * tx, ah);
                    load_center<R>(pv + (ty + R + d) * G::BX + 4 * tx, av);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        lh[k] = fmaf(cf.c[W + d + R], ah[k], lh[k]);
                        lv[k] = fmaf(cf.c[W + d + R], av[k], lv[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    // rho > 0 inside the grid; the guard keeps lanes past the edge finite
                    const float inv = rc[k] != 0.f ? 1.f / rc[k] : 0.f;
                    qh[R][k] = fmaf(rc[k], lh[k], qh[R][k]);
                    qv[R][k] = fmaf(inv, lv[k], qv[R][k]);
                }
            }
            if (zo >= 0) {
                const int o = ty * I::BXI + 4 * tx;
                load_center<I::OFF>(st + V::OFF_MV + o, mv);
                load_center<I::OFF>(st + V::OFF_RZ + o, rz);
                load_center<I::OFF>(st + V::OFF_HP + o, hp);
                load_center<I::OFF>(st + V::OFF_VP + o, vp);
                load_center<I::OFF>(st + V::OFF_HC + o, hc);
                load_center<I::OFF>(st + V::OFF_VC + o, vc);
            }
        } else {
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) return;
        if (tid == 0 && j + S < P) issue(j + S, s);
        if (zo >= 0) {
            const int z = zb + zo;
            const int y = y0 + ty;
            const float gzv = sponge(z, geo.nz, geo.sponge_w, geo.sponge_a);
            if (y < geo.ny && gx < geo.nx) {
                const int64_t mp = (int64_t)(z + R) * geo.pz + (int64_t)(y + R) * geo.py + (gx + R);
                float rh[4], rv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float g = gxs[k] * gys * gzv;
                    const bool at_src = gx + k == sx && y == sy && z == sz;
                    float a = 2.f * hc[k] + mv[k] * qh[0][k] - g * hp[k];
                    float b = 2.f * vc[k] + (mv[k] * rz[k]) * qv[0][k] - g * vp[k];
                    if (at_src) {
                        a += samp;
                        b += samp;
                    }
                    rh[k] = g * a;
                    rv[k] = g * b;
                }
                float *oh = hnext + shot_off + mp, *ov = vnext + shot_off + mp;
                if (vec && gx + 3 < geo.nx) {
                    *reinterpret_cast<float4 *>(oh) = make_float4(rh[0], rh[1], rh[2], rh[3]);
                    *reinterpret_cast<float4 *>(ov) = make_float4(rv[0], rv[1], rv[2], rv[3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (gx + k < geo.nx) {
                            oh[k] = rh[k];
                            ov[k] = rv[k];
                        }
                }
                if (rec && z == geo.rec_z) {
                    float *rp = rec + ((int64_t)sh * geo.ny + y) * geo.nx + gx;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (gx + k < geo.nx) rp[k] = rh[k];
                }
            }
        }
#pragma unroll
        for (int kk = 0; kk < W - 1; ++kk)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                qh[kk][k] = qh[kk + 1][k];
                qv[kk][k] = qv[kk + 1][k];
            }
#pragma unroll
        for (int k = 0; k < 4; ++k) qh[W - 1][k] = qv[W - 1][k] = 0.f;
    }
}

// mv = vp^2 s sqrt(1 + 2 delta), rho = (1 + 2 eps) / sqrt(1 + 2 delta) into
// padded fields (halo 0); vp, eps, delta dense interior arrays.
__global__ void vti_model_kernel(WaveGeo geo, const float *__restrict__ vp, const float *__restrict__ eps,
                                 const float *__restrict__ delta, float *__restrict__ mv,
                                 float *__restrict__ rho, float s)
{
    const int r = geo.r;
    const int64_t X = geo.nx + 2 * r, Y = geo.ny + 2 * r, Z = geo.nz + 2 * r;
    const int64_t total = X * Y * Z;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t xx = i % X, yy = (i / X) % Y, zz = i / (X * Y);
        const int64_t x = xx - r, y = yy - r, z = zz - r;
        float a = 0.f, b = 0.f;
        if (x >= 0 && x < geo.nx && y >= 0 && y < geo.ny && z >= 0 && z < geo.nz) {
            const int64_t q = (z * geo.ny + y) * geo.nx + x;
            const float v = vp[q];
            const float sd = sqrtf(1.f + 2.f * delta[q]);
            a = v * v * s * sd;
            b = (1.f + 2.f * eps[q]) / sd;
        }
        const int64_t o = zz * geo.pz + yy * geo.py + xx;
        mv[o] = a;
        rho[o] = b;
    }
}

// ------------------------------------------------------------------ TTI
//
// Per field f (p, then q) the derivative pass writes Lap f and H1 f:
//     H1 f = nx^2 f_xx + ny^2 f_yy + nz^2 f_zz + 2 nx ny f_xy + 2 ny nz f_yz + 2 nx nz f_xz
// with n = (sin th cos ph, sin th sin ph, cos th) the tilt axis.  The axis
// terms use the second-derivative row w2; a mixed term composes two
// first-derivative rows w1 (Sec. 4.7), and since composed first derivatives
// commute, f_xz = D_z (D_x f) and f_yz = D_z (D_y f): every arriving plane
// adds its D_x f, D_y f and centre value, weighted along z, to three register
// queues (f_xz, f_yz, f_zz).  The in-plane terms f_xx and f_yy come from the
// output's centre plane, which a ring of R + 3 planes still holds when the
// output completes, and f_xy = D_x (D_y f) from a ring of the last R + 1
// planes' D_y f, so no per-point value has to wait in registers for the
// tilt.  The tilt (nx, ny, nz) of the output point arrives by TMA (or by
// plain loads where rows are not 16-byte multiples).
//
// The q pass (or, for rows TMA cannot stage, a separate pointwise combine)
// applies the printed coupling with a = vpx^2, b = vpz^2, c = vpn^2,
// d = vsz^2 (all times dt^2/h^2) and alpha:
//     p'' = a H2p + alpha b H1q + d (H1p - alpha H1q)
//     q'' = c/alpha H2p + b H1q - d (H2p/alpha - H2q),     H2 = Lap - H1
// and the damped leapfrog update, source and receivers of the acoustic step.

struct TtiCoef {
    float w2[2 * kMaxR + 1];
    float w1[2 * kMaxR + 1];
};

// MODE 0: p or q pass, tilt by plain loads (rows TMA cannot stage);
// MODE 1: the same with the tilt tiles by TMA; MODE 2: the q pass with the
// combine fused in.
template <int R, int TX, int TY, int MODE>
struct TtiGeom {
    static constexpr bool FUSED = MODE == 2;
    using G = Geom<R, TX, TY, 1, R + 3>;
    using I = Interior<R, TX>;
    static constexpr int S = R + 3;  // planes j - R .. j + 2 resident at step j
    static constexpr int PL = (G::PLANE + 31) & ~31;
    // fused q pass: a 2-deep ring of the completing output's tiles --
    // 10 dense (Lap p, H1 p, a, b, c, d, alpha, nx, ny, nz) and 3 padded
    // interior tiles (p^n, p^{n-1}, q^{n-1})
    static constexpr int DT = (TX * TY + 31) & ~31;
    static constexpr int PT = (I::BXI * TY + 31) & ~31;
    static constexpr int CT = FUSED ? 10 * DT + 3 * PT : MODE == 1 ? 3 * DT : 0;
    static constexpr int CRING = MODE >= 1 ? 2 : 0;
    // D_y f of the last R + 1 planes, BX columns wide (the plane's column
    // indexing, x halo included) and TY rows: f_xy = D_x (D_y f) at completion
    static constexpr int DR = R + 1;
    static constexpr int DYT = (G::BX * TY + 31) & ~31;
    static constexpr size_t SMEM = 128 + ((size_t)S * PL + (size_t)CRING * CT + (size_t)DR * DYT) * 4 +
                                   (S + CRING) * sizeof(uint64_t) + 16;
    static_assert(SMEM <= 227 * 1024, "TTI rings exceed shared memory");
};

// Dense interior arrays (nshots stacked where per shot): x fastest.
struct TtiDense {
    int64_t sy, sz, ss;  // strides of y, z, shot (elements)
};

// What the fused q pass reads and writes besides the q planes.
struct TtiFused {
    CUtensorMap med;           // 8 dense fields (x, y, z, field)
    CUtensorMap work;          // Lap p, H1 p, ... slices (x, y, z, field * nshots + shot)
    CUtensorMap pc, pp, qp;    // padded interior tiles of p^n, p^{n-1}, q^{n-1}
    float *pn, *qn;
    const float *amp;
    float *rec;
};

// The arriving plane's contributions to the z queues: centre value (f_zz),
// D_x f (f_xz) and D_y f (f_yz), each weighted for the slot's offset.
template <int R, int NV, int BX, int NTX>
__device__ __forceinline__ void tti_arrive(const float *pl, const TtiCoef &cf, int tx, int ty,
                                           float (&qzz)[2 * R + 1][4], float (&qxz)[2 * R + 1][4],
                                           float (&qyz)[2 * R + 1][4], float *dyrow)
{
    constexpr int W = 2 * R + 1;
    float win[4 * NV];
    load_row<NV>(pl + (ty + R) * BX + 4 * tx, win);
    float dx[4], dy[4], c0[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        c0[k] = win[k + R];
        dx[k] = 0.f;
#pragma unroll
        for (int d = 1; d <= R; ++d)
            dx[k] = fmaf(cf.w1[R + d], win[k + R + d], fmaf(cf.w1[R - d], win[k + R - d], dx[k]));
        dy[k] = 0.f;
    }
#pragma unroll
    for (int d = -R; d <= R; ++d) {
        if (d == 0) continue;
        float a[4];
        load_center<R>(pl + (ty + R + d) * BX + 4 * tx, a);
#pragma unroll
        for (int k = 0; k < 4; ++k) dy[k] = fmaf(cf.w1[R + d], a[k], dy[k]);
    }
    // D_y f into the ring row at the plane's column indices; the x-halo
    // columns that f_xy's window reaches (R on each side) take one thread
    // each, the row's first 2R, so that a warp runs the halo sums once
    // instead of R times on two threads
#pragma unroll
    for (int k = 0; k < 4; ++k) dyrow[4 * tx + R + k] = dy[k];
    static_assert(NTX >= 2 * R, "a thread per x-halo column");
    if (tx < 2 * R) {
        const int c = tx < R ? tx : 4 * NTX + tx;  // 0 .. R-1, then 4 NTX + R .. 4 NTX + 2R - 1
        float v = 0.f;
#pragma unroll
        for (int d = -R; d <= R; ++d)
            if (d != 0) v = fmaf(cf.w1[R + d], pl[(ty + R + d) * BX + c], v);
        dyrow[c] = v;
    }
#pragma unroll
    for (int kk = 0; kk < W; ++kk)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int d = R - kk;  // offset of this plane from slot kk's output plane
            qzz[kk][k] = fmaf(cf.w2[R + d], c0[k], qzz[kk][k]);
            if (d != 0) {
                qxz[kk][k] = fmaf(cf.w1[R + d], dx[k], qxz[kk][k]);
                qyz[kk][k] = fmaf(cf.w1[R + d], dy[k], qyz[kk][k]);
            }
        }
}

// The in-plane terms of the output's centre plane: f_xx, f_yy, and f_xy as
// D_x of the plane's D_y f row (dyrow); also returns the centre values.
template <int R, int NV, int BX>
__device__ __forceinline__ void tti_centre(const float *pc, const float *dyrow, const TtiCoef &cf, int tx, int ty,
                                           float (&fxx)[4], float (&fyy)[4], float (&fxy)[4], float (&ctr)[4])
{
    float w[4 * NV], v[4 * NV];
    load_row<NV>(pc + (ty + R) * BX + 4 * tx, w);
    load_row<NV>(dyrow + 4 * tx, v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ctr[k] = w[k + R];
        fxx[k] = 0.f;
        fxy[k] = 0.f;
#pragma unroll
        for (int a = -R; a <= R; ++a) fxx[k] = fmaf(cf.w2[R + a], w[k + R + a], fxx[k]);
#pragma unroll
        for (int a = 1; a <= R; ++a)
            fxy[k] = fmaf(cf.w1[R + a], v[k + R + a], fmaf(cf.w1[R - a], v[k + R - a], fxy[k]));
        fyy[k] = cf.w2[R] * w[k + R];
    }
#pragma unroll
    for (int b = -R; b <= R; ++b) {
        if (b == 0) continue;
        float a[4];
        load_center<R>(pc + (ty + R + b) * BX + 4 * tx, a);
#pragma unroll
        for (int k = 0; k < 4; ++k) fyy[k] = fmaf(cf.w2[R + b], a[k], fyy[k]);
    }
}

__device__ __forceinline__ float tti_h1(float nx, float ny, float nz, float fxx, float fyy, float fzz, float fxy,
                                        float fxz, float fyz)
{
    float t = nx * nx * fxx;
    t = fmaf(ny * ny, fyy, t);
    t = fmaf(nz * nz, fzz, t);
    t = fmaf(2.f * nx * ny, fxy, t);
    t = fmaf(2.f * ny * nz, fyz, t);
    return fmaf(2.f * nx * nz, fxz, t);
}

// The derivative pass of one field (MODE 0 and 1: writes Lap f and H1 f),
// or the q pass with the combine fused in (MODE 2: reads Lap p, H1 p and the
// medium with the completing output's tiles, writes p^{n+1} and q^{n+1}).
template <int R, int TX, int TY, int MODE>
__global__ void __launch_bounds__(Geom<R, TX, TY, 1, R + 3>::NT)
    tti_deriv_kernel(const __grid_constant__ CUtensorMap tf, const __grid_constant__ TtiCoef cf,
                     const __grid_constant__ WaveGeo geo, const float *__restrict__ tilt, TtiDense dn,
                     float *__restrict__ lap, float *__restrict__ h1, const __grid_constant__ TtiFused fu,
                     int tz, int nzc, int vec, unsigned *err)
{
    using T = TtiGeom<R, TX, TY, MODE>;
    using G = typename T::G;
    using I = Interior<R, TX>;
    constexpr int W = G::W;
    constexpr int S = T::S;
    constexpr bool FUSED = T::FUSED;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_align128(smem_raw);
    float *planes = reinterpret_cast<float *>(smem);
    float *ctiles = planes + (size_t)S * T::PL;
    float *dyring = ctiles + (size_t)T::CRING * T::CT;
    uint64_t *full = reinterpret_cast<uint64_t *>(dyring + (size_t)T::DR * T::DYT);
    uint64_t *cfull = full + S;
    int &abort_flag = *reinterpret_cast<int *>(cfull + T::CRING);

    const int tid = threadIdx.x;
    const int tx = tid % G::NTX, ty = tid / G::NTX;
    const int sh = blockIdx.z / nzc, zc = blockIdx.z % nzc;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, zb = zc * tz;
    const int nzt = min(tz, geo.nz - zb);
    const int P = nzt + 2 * R;
    const int gx = x0 + 4 * tx, y = y0 + ty;
    const int64_t npts = (int64_t)geo.nz * dn.sz;  // one dense field

    auto issue = [&](int j) {
        const int s = j % S;
        ptx::mbar_arrive_expect_tx(&full[s], G::PLANE * 4);
        ptx::tma_load_4d(planes + (size_t)s * T::PL, &tf, x0, y0, zb + j, sh, &full[s]);
    };
    // fused: the tiles of output plane zo into completion slot zo % 2
    auto issue_c = [&](int zo) {
        if constexpr (MODE == 1) {
            const int c = zo % 2;
            float *ct = ctiles + (size_t)c * T::CT;
            ptx::mbar_arrive_expect_tx(&cfull[c], 3 * TX * TY * 4);
#pragma unroll
            for (int f = 0; f < 3; ++f) ptx::tma_load_4d(ct + f * T::DT, &fu.med, x0, y0, zb + zo, 5 + f, &cfull[c]);
        }
        if constexpr (FUSED) {
            const int c = zo % 2;
            float *ct = ctiles + (size_t)c * T::CT;
            ptx::mbar_arrive_expect_tx(&cfull[c], (10 * TX * TY + 3 * I::BXI * TY) * 4);
            const int z = zb + zo;
            ptx::tma_load_4d(ct + 0 * T::DT, &fu.work, x0, y0, z, sh, &cfull[c]);                // Lap p
            ptx::tma_load_4d(ct + 1 * T::DT, &fu.work, x0, y0, z, geo.nshots + sh, &cfull[c]);   // H1 p
#pragma unroll
            for (int f = 0; f < 8; ++f) ptx::tma_load_4d(ct + (2 + f) * T::DT, &fu.med, x0, y0, z, f, &cfull[c]);
            const int xs = x0 + (R & ~3), zp = z + R;
            ptx::tma_load_4d(ct + 10 * T::DT, &fu.pc, xs, y0 + R, zp, sh, &cfull[c]);
            ptx::tma_load_4d(ct + 10 * T::DT + T::PT, &fu.pp, xs, y0 + R, zp, sh, &cfull[c]);
            ptx::tma_load_4d(ct + 10 * T::DT + 2 * T::PT, &fu.qp, xs, y0 + R, zp, sh, &cfull[c]);
        }
    };
    if (tid == 0) {
        ptx::prefetch_tmap(&tf);
#pragma unroll
        for (int s = 0; s < S; ++s) ptx::mbar_init(&full[s], 1);
#pragma unroll
        for (int c = 0; c < T::CRING; ++c) ptx::mbar_init(&cfull[c], 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();
    if (tid == 0) {
        for (int j = 0; j < S && j < P; ++j) issue(j);
        if constexpr (MODE >= 1)
            for (int zo = 0; zo < 2 && zo < nzt; ++zo) issue_c(zo);
    }

    float gxs[4] = {1.f, 1.f, 1.f, 1.f}, gys = 1.f;
    if constexpr (FUSED) {
#pragma unroll
        for (int k = 0; k < 4; ++k) gxs[k] = sponge(gx + k, geo.nx, geo.sponge_w, geo.sponge_a);
        gys = sponge(y, geo.ny, geo.sponge_w, geo.sponge_a);
    }

    float qzz[W][4], qxz[W][4], qyz[W][4];
#pragma unroll
    for (int kk = 0; kk < W; ++kk)
#pragma unroll
        for (int k = 0; k < 4; ++k) qzz[kk][k] = qxz[kk][k] = qyz[kk][k] = 0.f;

    const bool inside = y < geo.ny && gx < geo.nx;
    for (int j = 0; j < P; ++j) {
        const int zo = j - 2 * R;
        // unfused: the output's tilt, read early so that its latency overlaps the plane work
        float n3[3][4] = {};
        if (MODE == 0 && zo >= 0 && inside) {
            const int64_t o = (int64_t)(zb + zo) * dn.sz + (int64_t)y * dn.sy + gx;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float *src = tilt + c * npts + o;
                if (vec) {
                    const float4 t = __ldg(reinterpret_cast<const float4 *>(src));
                    n3[c][0] = t.x; n3[c][1] = t.y; n3[c][2] = t.z; n3[c][3] = t.w;
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) n3[c][k] = gx + k < geo.nx ? __ldg(src + k) : 0.f;
                }
            }
        }
        const int s = j % S;
        float fxx[4], fyy[4], fxy[4], ctr[4];
        // fused completion values: Lap p, H1 p, a, b, c, d, alpha, nx, ny, nz, p^n, p^{n-1}, q^{n-1}
        float cv[13][4];
        bool ok = ptx::mbar_wait_bounded(&full[s], (uint32_t)(j / S) & 1u, err);
        if (ok) {
            tti_arrive<R, G::NV, G::BX, G::NTX>(planes + (size_t)s * T::PL, cf, tx, ty, qzz, qxz, qyz,
                                                dyring + (size_t)(j % T::DR) * T::DYT + ty * G::BX);
            if (zo >= 0) {
                // the centre plane j - R and its D_y f, stored R steps ago
                tti_centre<R, G::NV, G::BX>(planes + (size_t)((j - R) % S) * T::PL,
                                            dyring + (size_t)((j - R) % T::DR) * T::DYT + ty * G::BX, cf, tx, ty,
                                            fxx, fyy, fxy, ctr);
                if constexpr (MODE == 1) {
                    const int c = zo % 2;
                    ok = ptx::mbar_wait_bounded(&cfull[c], (uint32_t)(zo / 2) & 1u, err);
                    if (ok) {
                        const float *ct = ctiles + (size_t)c * T::CT;
#pragma unroll
                        for (int f = 0; f < 3; ++f) {
                            const float4 t = *reinterpret_cast<const float4 *>(ct + f * T::DT + ty * TX + 4 * tx);
                            n3[f][0] = t.x; n3[f][1] = t.y; n3[f][2] = t.z; n3[f][3] = t.w;
                        }
                    }
                }
                if constexpr (FUSED) {
                    const int c = zo % 2;
                    ok = ptx::mbar_wait_bounded(&cfull[c], (uint32_t)(zo / 2) & 1u, err);
                    if (ok) {
                        const float *ct = ctiles + (size_t)c * T::CT;
#pragma unroll
                        for (int f = 0; f < 10; ++f) {
                            const float4 t = *reinterpret_cast<const float4 *>(ct + f * T::DT + ty * TX + 4 * tx);
                            cv[f][0] = t.x; cv[f][1] = t.y; cv[f][2] = t.z; cv[f][3] = t.w;
                        }
#pragma unroll
                        for (int f = 0; f < 3; ++f)
                            load_center<I::OFF>(ct + 10 * T::DT + f * T::PT + ty * I::BXI + 4 * tx, cv[10 + f]);
                    }
                }
            }
        }
        if (!ok) abort_flag = 1;
        __syncthreads();
        if (abort_flag) return;
        // plane j - R is no longer needed: its stage takes plane j - R + S;
        // the completion slot of zo takes output zo + 2
        if (tid == 0) {
            if (j >= R && j - R + S < P) issue(j - R + S);
            if constexpr (MODE >= 1)
                if (zo >= 0 && zo + 2 < nzt) issue_c(zo + 2);
        }
        if (zo >= 0 && inside) {
            if constexpr (!FUSED) {
                float l[4], h[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    l[k] = fxx[k] + fyy[k] + qzz[0][k];
                    h[k] = tti_h1(n3[0][k], n3[1][k], n3[2][k], fxx[k], fyy[k], qzz[0][k], fxy[k], qxz[0][k],
                                  qyz[0][k]);
                }
                const int64_t o = (int64_t)sh * dn.ss + (int64_t)(zb + zo) * dn.sz + (int64_t)y * dn.sy + gx;
                if (vec) {
                    *reinterpret_cast<float4 *>(lap + o) = make_float4(l[0], l[1], l[2], l[3]);
                    *reinterpret_cast<float4 *>(h1 + o) = make_float4(h[0], h[1], h[2], h[3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (gx + k < geo.nx) {
                            lap[o + k] = l[k];
                            h1[o + k] = h[k];
                        }
                }
            } else {
                const int z = zb + zo;
                const float gzy = gys * sponge(z, geo.nz, geo.sponge_w, geo.sponge_a);
                const float samp = fu.amp[sh];
                const int sx = geo.src[sh][0], sy = geo.src[sh][1], sz = geo.src[sh][2];
                float rp4[4], rq4[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float H1q = tti_h1(cv[7][k], cv[8][k], cv[9][k], fxx[k], fyy[k], qzz[0][k], fxy[k],
                                             qxz[0][k], qyz[0][k]);
                    const float H2q = fxx[k] + fyy[k] + qzz[0][k] - H1q;
                    const float H1p = cv[1][k], H2p = cv[0][k] - H1p;
                    const float a = cv[2][k], b = cv[3][k], c = cv[4][k], d = cv[5][k], al = cv[6][k];
                    const float inv = al != 0.f ? 1.f / al : 0.f;  // alpha > 0 inside the grid
                    const float rp = a * H2p + al * b * H1q + d * (H1p - al * H1q);
                    const float rq = c * inv * H2p + b * H1q - d * (H2p * inv - H2q);
                    const float g = gxs[k] * gzy;
                    const float sv = (gx + k == sx && y == sy && z == sz) ? samp : 0.f;
                    rp4[k] = g * (2.f * cv[10][k] - g * cv[11][k] + rp + sv);
                    rq4[k] = g * (2.f * ctr[k] - g * cv[12][k] + rq + sv);
                }
                const int64_t mp = (int64_t)sh * geo.ss + (int64_t)(z + R) * geo.pz + (int64_t)(y + R) * geo.py +
                                   (gx + R);
                float *op = fu.pn + mp, *oq = fu.qn + mp;
                if (vec && R % 4 == 0 && gx + 3 < geo.nx) {
                    *reinterpret_cast<float4 *>(op) = make_float4(rp4[0], rp4[1], rp4[2], rp4[3]);
                    *reinterpret_cast<float4 *>(oq) = make_float4(rq4[0], rq4[1], rq4[2], rq4[3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (gx + k < geo.nx) {
                            op[k] = rp4[k];
                            oq[k] = rq4[k];
                        }
                }
                if (fu.rec && z == geo.rec_z) {
                    float *rp = fu.rec + ((int64_t)sh * geo.ny + y) * geo.nx + gx;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (gx + k < geo.nx) rp[k] = rp4[k];
                }
            }
        }
#pragma unroll
        for (int kk = 0; kk < W - 1; ++kk)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                qzz[kk][k] = qzz[kk + 1][k];
                qxz[kk][k] = qxz[kk + 1][k];
                qyz[kk][k] = qyz[kk + 1][k];
            }
#pragma unroll
        for (int k = 0; k < 4; ++k) qzz[W - 1][k] = qxz[W - 1][k] = qyz[W - 1][k] = 0.f;
    }
}

// Pointwise combine: one thread per (shot, z, y, 4 x).  med: 5 dense
// interior fields (a, b, c, d, alpha); work: Lap p, H1 p, Lap q, H1 q.
__global__ void tti_combine_kernel(WaveGeo geo, TtiDense dn, const float *__restrict__ med,
                                   const float *__restrict__ lp, const float *__restrict__ hp,
                                   const float *__restrict__ lq, const float *__restrict__ hq,
                                   const float *__restrict__ pc, const float *__restrict__ qc,
                                   const float *__restrict__ pp, const float *__restrict__ qp,
                                   float *__restrict__ pn, float *__restrict__ qn,
                                   const float *__restrict__ amp, float *__restrict__ rec)
{
    const int r = geo.r;
    const int nxq = (geo.nx + 3) / 4;
    const int64_t per_shot = (int64_t)geo.nz * geo.ny * nxq;
    const int64_t total = per_shot * geo.nshots;
    const int64_t npts = (int64_t)geo.nz * dn.sz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int sh = (int)(i / per_shot);
        const int64_t rem = i % per_shot;
        const int xq = (int)(rem % nxq);
        const int y = (int)((rem / nxq) % geo.ny);
        const int z = (int)(rem / ((int64_t)nxq * geo.ny));
        const float gy = sponge(y, geo.ny, geo.sponge_w, geo.sponge_a) * sponge(z, geo.nz, geo.sponge_w, geo.sponge_a);
        const float s_amp = amp[sh];
        const int64_t od = (int64_t)z * dn.sz + (int64_t)y * dn.sy;
        const int64_t ow = (int64_t)sh * dn.ss + od;
        const int64_t of = (int64_t)sh * geo.ss + (int64_t)(z + r) * geo.pz + (int64_t)(y + r) * geo.py + r;
        for (int k = 0; k < 4; ++k) {
            const int x = 4 * xq + k;
            if (x >= geo.nx) break;
            const float a = med[od + x], b = med[npts + od + x], c = med[2 * npts + od + x];
            const float d = med[3 * npts + od + x], al = med[4 * npts + od + x];
            const float H1p = hp[ow + x], H1q = hq[ow + x];
            const float H2p = lp[ow + x] - H1p, H2q = lq[ow + x] - H1q;
            const float inv = 1.f / al;
            const float rp = a * H2p + al * b * H1q + d * (H1p - al * H1q);
            const float rq = c * inv * H2p + b * H1q - d * (H2p * inv - H2q);
            const float g = sponge(x, geo.nx, geo.sponge_w, geo.sponge_a) * gy;
            const bool at_src = x == geo.src[sh][0] && y == geo.src[sh][1] && z == geo.src[sh][2];
            const float s = at_src ? s_amp : 0.f;
            const float vp = g * (2.f * pc[of + x] - g * pp[of + x] + rp + s);
            const float vq = g * (2.f * qc[of + x] - g * qp[of + x] + rq + s);
            pn[of + x] = vp;
            qn[of + x] = vq;
            if (rec && z == geo.rec_z) rec[((int64_t)sh * geo.ny + y) * geo.nx + x] = vp;
        }
    }
}

// The medium of the TTI step from the Thomsen parameters: 8 dense interior
// fields [a, b, c, d, alpha, nx, ny, nz] with a = vp^2 (1+2 eps) s,
// b = vp^2 s, c = vp^2 (1+2 delta) s, d = vs^2 s (s = dt^2/h^2).
__global__ void tti_model_kernel(int64_t n, const float *__restrict__ vp, const float *__restrict__ vs,
                                 const float *__restrict__ eps, const float *__restrict__ delta,
                                 const float *__restrict__ alpha, const float *__restrict__ theta,
                                 const float *__restrict__ phi, float *__restrict__ med, float s)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v2 = vp[i] * vp[i] * s;
        float st, ct, sp, cp;
        sincosf(theta[i], &st, &ct);
        sincosf(phi[i], &sp, &cp);
        med[i] = v2 * (1.f + 2.f * eps[i]);
        med[n + i] = v2;
        med[2 * n + i] = v2 * (1.f + 2.f * delta[i]);
        med[3 * n + i] = vs[i] * vs[i] * s;
        med[4 * n + i] = alpha[i];
        med[5 * n + i] = st * cp;
        med[6 * n + i] = st * sp;
        med[7 * n + i] = ct;
    }
}

constexpr int kTtiTX = 64, kTtiTY = 8, kTtiTZ = 128;

template <int R, int MODE>
cudaError_t tti_deriv_r(const WaveGeo &g, const TtiCoef &cf, const float *f, const float *tilt, TtiDense dn,
                        float *lap, float *h1, const TtiFused &fu, cudaStream_t st)
{
    using T = TtiGeom<R, kTtiTX, kTtiTY, MODE>;
    using G = typename T::G;
    const int X = g.nx + 2 * R, Y = g.ny + 2 * R, Z = g.nz + 2 * R;
    CUtensorMap tf;
    if (!encode_tmap_4d(&tf, f, X, Y, Z, g.nshots, g.py, g.pz, g.ss, G::BX, G::BY, 1))
        return cudaErrorInvalidValue;
    auto kern = tti_deriv_kernel<R, kTtiTX, kTtiTY, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
    if (e != cudaSuccess) return e;
    const int tz = kTtiTZ;
    const int nzc = (g.nz + tz - 1) / tz;
    const dim3 grid((g.nx + kTtiTX - 1) / kTtiTX, (g.ny + kTtiTY - 1) / kTtiTY, nzc * g.nshots);
    int vec = g.nx % 4 == 0 && reinterpret_cast<uintptr_t>(tilt) % 16 == 0 &&
              reinterpret_cast<uintptr_t>(lap) % 16 == 0 && reinterpret_cast<uintptr_t>(h1) % 16 == 0;
    if (MODE == 2)
        vec = g.py % 4 == 0 && g.pz % 4 == 0 && g.ss % 4 == 0 && reinterpret_cast<uintptr_t>(fu.pn) % 16 == 0 &&
              reinterpret_cast<uintptr_t>(fu.qn) % 16 == 0;
    kern<<<grid, G::NT, T::SMEM, st>>>(tf, cf, g, tilt, dn, lap, h1, fu, tz, nzc, vec, device_error_word());
    return cudaGetLastError();
}

template <int MODE>
cudaError_t tti_deriv(const WaveGeo &g, const TtiCoef &cf, const float *f, const float *tilt, TtiDense dn,
                      float *lap, float *h1, const TtiFused &fu, cudaStream_t st)
{
    switch (g.r) {
        case 1: return tti_deriv_r<1, MODE>(g, cf, f, tilt, dn, lap, h1, fu, st);
        case 2: return tti_deriv_r<2, MODE>(g, cf, f, tilt, dn, lap, h1, fu, st);
        case 3: return tti_deriv_r<3, MODE>(g, cf, f, tilt, dn, lap, h1, fu, st);
        case 4: return tti_deriv_r<4, MODE>(g, cf, f, tilt, dn, lap, h1, fu, st);
        default: return cudaErrorInvalidValue;
    }
}

// Tensor maps of the fused q pass (dense maps need nx % 4 == 0: 16-byte rows).
template <int R>
bool tti_fused_maps(const WaveGeo &g, const float *med, const float *work, const float *pc, const float *pp,
                    const float *qp, TtiFused *fu)
{
    using I = Interior<R, kTtiTX>;
    const int X = g.nx + 2 * R, Y = g.ny + 2 * R, Z = g.nz + 2 * R;
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny, n = sz * g.nz;
    return encode_tmap_4d(&fu->med, med, g.nx, g.ny, g.nz, 8, sy, sz, n, kTtiTX, kTtiTY, 1) &&
           encode_tmap_4d(&fu->work, work, g.nx, g.ny, g.nz, 2 * g.nshots, sy, sz, n, kTtiTX, kTtiTY, 1) &&
           encode_tmap_4d(&fu->pc, pc, X, Y, Z, g.nshots, g.py, g.pz, g.ss, I::BXI, kTtiTY, 1) &&
           encode_tmap_4d(&fu->pp, pp, X, Y, Z, g.nshots, g.py, g.pz, g.ss, I::BXI, kTtiTY, 1) &&
           encode_tmap_4d(&fu->qp, qp, X, Y, Z, g.nshots, g.py, g.pz, g.ss, I::BXI, kTtiTY, 1);
}

// Tile variants of the VTI step: (TX, TY, stages, z chunk).
struct VtiVariant { int tx, ty, s, tz; };
// Variant 0 is the default (fastest on GB300 for 4 shots x 512^3, r = 4).
constexpr VtiVariant kVtiVariants[] = {{64, 8, 3, 256}, {64, 16, 2, 128}, {32, 16, 3, 128}, {64, 16, 3, 128},
                                       {64, 8, 4, 128}, {64, 8, 3, 128}, {128, 8, 2, 128}, {32, 8, 3, 128},
                                       {64, 8, 2, 128}};
constexpr int kNumVtiVariants = sizeof(kVtiVariants) / sizeof(kVtiVariants[0]);
int g_vti_variant = 0;

template <int R, int TX, int TY, int S>
cudaError_t vti_launch(const WaveGeo &g, const StarCoef &cf, int tz, const float *mv, const float *rho,
                       const float *hcur, const float *vcur, const float *hprev, const float *vprev, float *hnext,
                       float *vnext, const float *amp, float *rec, cudaStream_t st)
{
    using G = Geom<R, TX, TY, 1, S>;
    using V = VtiGeom<R, TX, TY, S>;
    using I = Interior<R, TX>;
    const int X = g.nx + 2 * R, Y = g.ny + 2 * R, Z = g.nz + 2 * R;
    VtiMaps tm;
    if (!encode_tmap_4d(&tm.h, hcur, X, Y, Z, g.nshots, g.py, g.pz, g.ss, G::BX, G::BY, 1) ||
        !encode_tmap_4d(&tm.v, vcur, X, Y, Z, g.nshots, g.py, g.pz, g.ss, G::BX, G::BY, 1) ||
        !encode_tmap_3d(&tm.rho, rho, X, Y, Z, g.py, g.pz, I::BXI, TY, 1) ||
        !encode_tmap_3d(&tm.mv, mv, X, Y, Z, g.py, g.pz, I::BXI, TY, 1) ||
        !encode_tmap_4d(&tm.hp, hprev, X, Y, Z, g.nshots, g.py, g.pz, g.ss, I::BXI, TY, 1) ||
        !encode_tmap_4d(&tm.vp, vprev, X, Y, Z, g.nshots, g.py, g.pz, g.ss, I::BXI, TY, 1) ||
        !encode_tmap_4d(&tm.hc, hcur, X, Y, Z, g.nshots, g.py, g.pz, g.ss, I::BXI, TY, 1) ||
        !encode_tmap_4d(&tm.vc, vcur, X, Y, Z, g.nshots, g.py, g.pz, g.ss, I::BXI, TY, 1))
        return cudaErrorInvalidValue;
    auto kern = vti_fwd_kernel<R, TX, TY, S>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)V::SMEM);
    if (e != cudaSuccess) return e;
    const int nzc = (g.nz + tz - 1) / tz;
    const dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, nzc * g.nshots);
    const int vec = (R % 4 == 0) && g.py % 4 == 0 && g.pz % 4 == 0 && g.ss % 4 == 0 &&
                    reinterpret_cast<uintptr_t>(hnext) % 16 == 0 && reinterpret_cast<uintptr_t>(vnext) % 16 == 0;
    kern<<<grid, G::NT, V::SMEM, st>>>(tm, cf, g, hnext, vnext, amp, rec, tz, nzc, vec, device_error_word());
    return cudaGetLastError();
}

template <int R>
cudaError_t vti_r(int variant, const WaveGeo &g, const StarCoef &cf, const float *mv, const float *rho,
                  const float *hcur, const float *vcur, const float *hprev, const float *vprev, float *hnext,
                  float *vnext, const float *amp, float *rec, cudaStream_t st)
{
    const VtiVariant v = kVtiVariants[variant];
#define MMS_VTI_CASE(TX_, TY_, S_)                                                                          \
    if (v.tx == TX_ && v.ty == TY_ && v.s == S_)                                                            \
        return vti_launch<R, TX_, TY_, S_>(g, cf, v.tz, mv, rho, hcur, vcur, hprev, vprev, hnext, vnext, amp, \
                                           rec, st);
    MMS_VTI_CASE(64, 8, 3)
    MMS_VTI_CASE(64, 16, 2)
    MMS_VTI_CASE(32, 16, 3)
    MMS_VTI_CASE(64, 16, 3)
    MMS_VTI_CASE(64, 8, 4)
    MMS_VTI_CASE(128, 8, 2)
    MMS_VTI_CASE(32, 8, 3)
    MMS_VTI_CASE(64, 8, 2)
#undef MMS_VTI_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

int vti_num_variants() { return kNumVtiVariants; }

bool vti_set_variant(int v)
{
    if (v < 0 || v >= kNumVtiVariants) return false;
    g_vti_variant = v;
    return true;
}

cudaError_t launch_vti_step(const WaveGeo &g, const float *coeffs, const float *mv, const float *rho,
                            const float *hcur, const float *vcur, const float *hprev, const float *vprev,
                            float *hnext, float *vnext, const float *src_amp, float *rec, cudaStream_t st)
{
    StarCoef cf{};
    for (int i = 0; i < 3 * (2 * g.r + 1); ++i) cf.c[i] = coeffs[i];
    const int v = g_vti_variant;
    switch (g.r) {
        case 1: return vti_r<1>(v, g, cf, mv, rho, hcur, vcur, hprev, vprev, hnext, vnext, src_amp, rec, st);
        case 2: return vti_r<2>(v, g, cf, mv, rho, hcur, vcur, hprev, vprev, hnext, vnext, src_amp, rec, st);
        case 3: return vti_r<3>(v, g, cf, mv, rho, hcur, vcur, hprev, vprev, hnext, vnext, src_amp, rec, st);
        case 4: return vti_r<4>(v, g, cf, mv, rho, hcur, vcur, hprev, vprev, hnext, vnext, src_amp, rec, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tti_step(const WaveGeo &g, const float *w2, const float *w1, const float *med,
                            const float *pc, const float *qc, const float *pp, const float *qp, float *pn, float *qn,
                            float *work, const float *src_amp, float *rec, cudaStream_t st)
{
    TtiCoef cf{};
    for (int i = 0; i < 2 * g.r + 1; ++i) {
        cf.w2[i] = w2[i];
        cf.w1[i] = w1[i];
    }
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    TtiDense dn{g.nx, (int64_t)g.nx * g.ny, n};
    float *lp = work, *hp = work + g.nshots * n, *lq = work + 2 * g.nshots * n, *hq = work + 3 * g.nshots * n;
    const float *tilt = med + 5 * n;
    TtiFused fu{};
    // Rows of 16 bytes (nx % 4 == 0): the p pass with its tilt by TMA, then
    // the q pass with the combine fused in (two launches).  Otherwise a p
    // pass and a q pass with plain tilt loads and a separate combine.
    if (g.nx % 4 == 0) {
        bool ok = false;
        switch (g.r) {
            case 1: ok = tti_fused_maps<1>(g, med, work, pc, pp, qp, &fu); break;
            case 2: ok = tti_fused_maps<2>(g, med, work, pc, pp, qp, &fu); break;
            case 3: ok = tti_fused_maps<3>(g, med, work, pc, pp, qp, &fu); break;
            case 4: ok = tti_fused_maps<4>(g, med, work, pc, pp, qp, &fu); break;
            default: return cudaErrorInvalidValue;
        }
        if (!ok) return cudaErrorInvalidValue;
        cudaError_t e = tti_deriv<1>(g, cf, pc, tilt, dn, lp, hp, fu, st);
        if (e != cudaSuccess) return e;
        fu.pn = pn;
        fu.qn = qn;
        fu.amp = src_amp;
        fu.rec = rec;
        return tti_deriv<2>(g, cf, qc, tilt, dn, nullptr, nullptr, fu, st);
    }
    cudaError_t e = tti_deriv<0>(g, cf, pc, tilt, dn, lp, hp, fu, st);
    if (e != cudaSuccess) return e;
    e = tti_deriv<0>(g, cf, qc, tilt, dn, lq, hq, fu, st);
    if (e != cudaSuccess) return e;
    tti_combine_kernel<<<152 * 8, 256, 0, st>>>(g, dn, med, lp, hp, lq, hq, pc, qc, pp, qp, pn, qn, src_amp, rec);
    return cudaGetLastError();
}

cudaError_t launch_tti_model(int64_t n, const float *vp, const float *vs, const float *eps, const float *delta,
                             const float *alpha, const float *theta, const float *phi, float *med, float dt, float h,
                             cudaStream_t st)
{
    const float s = (dt * dt) / (h * h);
    tti_model_kernel<<<152 * 8, 256, 0, st>>>(n, vp, vs, eps, delta, alpha, theta, phi, med, s);
    return cudaGetLastError();
}

cudaError_t launch_vti_model(const WaveGeo &g, const float *vp, const float *eps, const float *delta, float *mv,
                             float *rho, float dt, float h, cudaStream_t st)
{
    const float s = (dt * dt) / (h * h);
    vti_model_kernel<<<152 * 8, 256, 0, st>>>(g, vp, eps, delta, mv, rho, s);
    return cudaGetLastError();
}

}  // namespace mms
