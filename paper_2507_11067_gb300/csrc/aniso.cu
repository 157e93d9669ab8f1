// aniso.cu -- fused wave steps of the coupled anisotropic systems of the
// paper's Sec. 2.1: VTI (two stresses sigma_H, sigma_V).
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

// Tile variants of the VTI step: (TX, TY, stages, z chunk).
struct VtiVariant { int tx, ty, s, tz; };
// Variant 0 is the default (fastest on GB300 for 4 shots x 512^3, r = 4).
constexpr VtiVariant kVtiVariants[] = {{64, 8, 3, 128}, {64, 16, 2, 128}, {32, 16, 3, 128}, {64, 16, 3, 128},
                                       {64, 8, 4, 128}, {64, 8, 3, 256}, {128, 8, 2, 128}, {32, 8, 3, 128},
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

cudaError_t launch_vti_model(const WaveGeo &g, const float *vp, const float *eps, const float *delta, float *mv,
                             float *rho, float dt, float h, cudaStream_t st)
{
    const float s = (dt * dt) / (h * h);
    vti_model_kernel<<<152 * 8, 256, 0, st>>>(g, vp, eps, delta, mv, rho, s);
    return cudaGetLastError();
}

}  // namespace mms
