// sweep_cc.cu -- FP32 CUDA-core stencil sweeps for sm_103a.
//
// Star and box sweeps of the paper's Sec. 1 (Fig. 1), computed the GB300
// way rather than with the paper's CPU outer-product units:
//  * each CTA owns a TX x TY column of output points and marches a range of
//    TZ planes along z (2.5D blocking, the analogue of the paper's Sec. 4.5
//    per-core tiles marching the outer dimension);
//  * every input plane of the column plus its r-halo, (TX+2r) x (TY+2r)
//    floats, is staged in shared memory by one TMA bulk-tensor copy into an
//    S-deep mbarrier ring (the analogue of the paper's Sec. 4.4 brick layout
//    and gather prefetch: few, long, asynchronous streams);
//  * when plane j arrives it is consumed once: it adds its z-contribution
//    to the 2r+1 output planes it touches (a register queue of partial sums
//    per point) and, for the star, its in-plane x/y part to the output plane
//    it centres; the partial sum of the oldest plane is then complete and
//    leaves with float4 stores;
//  * the box adds, for each of the 2r+1 output planes, the 2D (2r+1)^2
//    stencil of weights c[dz] (the paper's Sec. 4.3 box decomposition into
//    per-plane stencils).
// Weights are kernel parameters, i.e. uniform constant-bank operands of the
// FMAs.  The naive kernel (one thread per point, global loads) serves any
// pitch and is the reference path of the library's own tests.
#include <stdio.h>

#include "common.cuh"
#include "tile.cuh"

namespace mms {
namespace {

// ---------------------------------------------------------------- naive
__global__ void naive_kernel(int shape, int r, const __grid_constant__ BoxCoef cf,
                             const float *__restrict__ in, int64_t ipy, int64_t ipz,
                             float *__restrict__ out, int64_t opy, int64_t opz, int64_t nx,
                             int64_t ny, int64_t nz)
{
    const int w = 2 * r + 1;
    const int64_t total = nx * ny * nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
        const float *c0 = in + (z + r) * ipz + (y + r) * ipy + (x + r);
        float acc = 0.f;
        if (shape == MMS_STAR) {
            for (int d = -r; d <= r; ++d) {
                acc = fmaf(cf.c[0 * w + d + r], c0[d], acc);
                acc = fmaf(cf.c[1 * w + d + r], c0[d * ipy], acc);
                acc = fmaf(cf.c[2 * w + d + r], c0[d * ipz], acc);
            }
        } else {
            for (int dz = -r; dz <= r; ++dz)
                for (int dy = -r; dy <= r; ++dy)
                    for (int dx = -r; dx <= r; ++dx)
                        acc = fmaf(cf.c[((dz + r) * w + dy + r) * w + dx + r],
                                   c0[dz * ipz + dy * ipy + dx], acc);
        }
        out[z * opz + y * opy + x] = acc;
    }
}

template <int R, int TX, int TY, int PY, int S, bool BOX, typename Coef>
__global__ void __launch_bounds__(Geom<R, TX, TY, PY, S>::NT)
    sweep_cc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ Coef cf,
                    float *__restrict__ out, int nx, int ny, int nz, int64_t opy, int64_t opz,
                    int tz, int vec_store, unsigned *err)
{
    using G = Geom<R, TX, TY, PY, S>;
    constexpr int W = G::W;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_align128(smem_raw);
    float *planes = reinterpret_cast<float *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)S * G::STAGE * sizeof(float));
    int &abort_flag = *reinterpret_cast<int *>(full + S);

    const int tid = threadIdx.x;
    const int tx = tid % G::NTX, ty = tid / G::NTX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, zb = blockIdx.z * tz;
    const int nzt = min(tz, nz - zb);
    const int P = nzt + 2 * R;  // padded planes this CTA consumes
    const int ry0 = ty * PY;
    const int gx = x0 + 4 * tx;

    if (tid == 0) {
        ptx::prefetch_tmap(&tmap);
#pragma unroll
        for (int s = 0; s < S; ++s) ptx::mbar_init(&full[s], 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();
    if (tid == 0) {
        for (int j = 0; j < S && j < P; ++j) {
            ptx::mbar_arrive_expect_tx(&full[j], G::PLANE * sizeof(float));
            ptx::tma_load_3d(planes + j * G::STAGE, &tmap, x0, y0, zb + j, &full[j]);
        }
    }

    float acc[W][PY][4];
#pragma unroll
    for (int kk = 0; kk < W; ++kk)
#pragma unroll
        for (int i = 0; i < PY; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[kk][i][k] = 0.f;

    for (int j = 0; j < P; ++j) {
        const int s = j % S;
        if (ptx::mbar_wait_bounded(&full[s], (uint32_t)(j / S) & 1u, err)) {
            const float *pl = planes + s * G::STAGE;
            if constexpr (BOX)
                box_plane<R, PY, G::BX, G::NV>(pl, cf, acc, tx, ry0);
            else {
                float ctr[PY][4];
                star_plane<R, PY, G::BX, G::NV>(pl, cf, acc, ctr, tx, ry0);
            }
        } else {
            abort_flag = 1;
        }
        __syncthreads();  // every thread is done with stage s
        if (abort_flag) return;
        if (tid == 0 && j + S < P) {
            ptx::mbar_arrive_expect_tx(&full[s], G::PLANE * sizeof(float));
            ptx::tma_load_3d(planes + s * G::STAGE, &tmap, x0, y0, zb + j + S, &full[s]);
        }
        const int zo = j - 2 * R;  // output plane completed by plane j
        if (zo >= 0) {
            const int64_t zoff = (int64_t)(zb + zo) * opz;
#pragma unroll
            for (int i = 0; i < PY; ++i) {
                const int y = y0 + ry0 + i;
                if (y < ny && gx < nx) {
                    float *o = out + zoff + (int64_t)y * opy + gx;
                    if (vec_store && gx + 3 < nx) {
                        *reinterpret_cast<float4 *>(o) =
                            make_float4(acc[0][i][0], acc[0][i][1], acc[0][i][2], acc[0][i][3]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (gx + k < nx) o[k] = acc[0][i][k];
                    }
                }
            }
        }
#pragma unroll
        for (int kk = 0; kk < W - 1; ++kk)
#pragma unroll
            for (int i = 0; i < PY; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[kk][i][k] = acc[kk + 1][i][k];
#pragma unroll
        for (int i = 0; i < PY; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[W - 1][i][k] = 0.f;
    }
}

struct Variant { int tx, ty, py, s, tz; };

// Tile variants (TX, TY, PY, stages, TZ) of the CUDA-core sweeps.
constexpr Variant kStarVariants[] = {
    {64, 32, 2, 4, 128}, {64, 16, 2, 4, 128}, {128, 16, 2, 4, 128}, {64, 32, 4, 3, 128},
    {64, 32, 2, 4, 64},  {128, 32, 2, 3, 64}, {64, 16, 1, 3, 128}, {64, 16, 1, 4, 256},
};
constexpr Variant kBoxVariants[] = {
    {64, 16, 2, 3, 64}, {64, 32, 2, 3, 64}, {32, 16, 2, 3, 64}, {64, 16, 4, 3, 64},
    {64, 8, 2, 3, 128}, {128, 16, 2, 3, 32}, {64, 16, 1, 3, 128}, {64, 8, 1, 3, 128},
};
constexpr int kNumStar = sizeof(kStarVariants) / sizeof(Variant);
constexpr int kNumBox = sizeof(kBoxVariants) / sizeof(Variant);

template <int R, int TX, int TY, int PY, int S, bool BOX, typename Coef>
cudaError_t launch_tiled(const Sweep &sw, const CUtensorMap &tmap, const Coef &cf, int tz)
{
    using G = Geom<R, TX, TY, PY, S>;
    auto kern = sweep_cc_kernel<R, TX, TY, PY, S, BOX, Coef>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((sw.nx + TX - 1) / TX), (unsigned)((sw.ny + TY - 1) / TY),
                    (unsigned)((sw.nz + tz - 1) / tz));
    const int vec = ((sw.opy % 4) == 0 && (sw.opz % 4) == 0 &&
                     (reinterpret_cast<uintptr_t>(sw.out) % 16) == 0)
                        ? 1
                        : 0;
    kern<<<grid, G::NT, G::SMEM, sw.stream>>>(tmap, cf, sw.out, (int)sw.nx, (int)sw.ny,
                                               (int)sw.nz, sw.opy, sw.opz, tz, vec,
                                               device_error_word());
    return cudaGetLastError();
}

template <int R, bool BOX, typename Coef>
cudaError_t dispatch_variant(const Sweep &sw, const CUtensorMap &tmap, const Coef &cf, int v)
{
    const Variant *tab = BOX ? kBoxVariants : kStarVariants;
    const int tz = tab[v].tz;
#define MMS_CASE(I)                                                                          \
    case I:                                                                                  \
        return launch_tiled<R, (BOX ? kBoxVariants : kStarVariants)[I].tx,                   \
                            (BOX ? kBoxVariants : kStarVariants)[I].ty,                      \
                            (BOX ? kBoxVariants : kStarVariants)[I].py,                      \
                            (BOX ? kBoxVariants : kStarVariants)[I].s, BOX, Coef>(sw, tmap, cf, \
                                                                                   tz);
    switch (v) {
        MMS_CASE(0)
        MMS_CASE(1)
        MMS_CASE(2)
        MMS_CASE(3)
        MMS_CASE(4)
        MMS_CASE(5)
        MMS_CASE(6)
        MMS_CASE(7)
        default: return cudaErrorInvalidValue;
    }
#undef MMS_CASE
}

}  // namespace

int star_cc_variants() { return kNumStar; }
int box_cc_variants() { return kNumBox; }

void star_cc_box(int r, int v, int *bx, int *by)
{
    const Variant &t = kStarVariants[v];
    *bx = (t.tx + 2 * r + 3) & ~3;
    *by = t.ty + 2 * r;
}

void box_cc_box(int r, int v, int *bx, int *by)
{
    const Variant &t = kBoxVariants[v];
    *bx = (t.tx + 2 * r + 3) & ~3;
    *by = t.ty + 2 * r;
}

cudaError_t launch_naive(const Sweep &s)
{
    BoxCoef cf{};
    const int w = 2 * s.r + 1;
    const int n = s.shape == MMS_STAR ? 3 * w : w * w * w;
    for (int i = 0; i < n; ++i) cf.c[i] = s.coeffs[i];
    const int64_t total = s.nx * s.ny * s.nz;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    naive_kernel<<<blocks, 256, 0, s.stream>>>(s.shape, s.r, cf, s.in, s.ipy, s.ipz, s.out, s.opy,
                                              s.opz, s.nx, s.ny, s.nz);
    return cudaGetLastError();
}

cudaError_t launch_star_cc(const Sweep &s, const CUtensorMap &tmap, int v)
{
    StarCoef cf{};
    const int w = 2 * s.r + 1;
    for (int i = 0; i < 3 * w; ++i) cf.c[i] = s.coeffs[i];
    switch (s.r) {
        case 1: return dispatch_variant<1, false>(s, tmap, cf, v);
        case 2: return dispatch_variant<2, false>(s, tmap, cf, v);
        case 3: return dispatch_variant<3, false>(s, tmap, cf, v);
        case 4: return dispatch_variant<4, false>(s, tmap, cf, v);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_box_cc(const Sweep &s, const CUtensorMap &tmap, int v)
{
    BoxCoef cf{};
    const int w = 2 * s.r + 1;
    for (int i = 0; i < w * w * w; ++i) cf.c[i] = s.coeffs[i];
    switch (s.r) {
        case 1: return dispatch_variant<1, true>(s, tmap, cf, v);
        case 2: return dispatch_variant<2, true>(s, tmap, cf, v);
        case 3: return dispatch_variant<3, true>(s, tmap, cf, v);
        case 4: return dispatch_variant<4, true>(s, tmap, cf, v);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mms
