// sweep_2d.cu -- FP32 CUDA-core sweeps of the planar stencils (Table I's 2D
// kernels: star2d, box2d) on nz independent planes padded in x and y.
//
// A CTA owns a TX-wide strip of one plane and marches down it in row blocks
// of TY outputs: block t, (TX+2r) x (TY+2r) floats, is staged by one TMA copy
// into an S-deep mbarrier ring, so the copies of the next blocks overlap the
// arithmetic of this one (the 2D analogue of the z-march of sweep_cc.cuh;
// with no third axis there is no register queue).  One thread waits for each
// staged block and the CTA barrier releases the others.  Weights are kernel
// parameters; outputs leave with float4 stores.
#include "common.cuh"
#include "tile.cuh"

namespace mms {
namespace {

template <int R, int TX, int TY, int PY, int S, bool BOX, typename Coef>
__global__ void __launch_bounds__(Geom<R, TX, TY, PY, S>::NT)
    plane_cc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ Coef cf,
                    float *__restrict__ out, int nx, int ny, int64_t opy, int64_t opz, int blocks_per_cta,
                    int vec_store, unsigned *err)
{
    using G = Geom<R, TX, TY, PY, S>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_align128(smem_raw);
    float *stages = reinterpret_cast<float *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)S * G::STAGE * sizeof(float));
    int &abort_flag = *reinterpret_cast<int *>(full + S);

    const int tid = threadIdx.x;
    const int tx = tid % G::NTX, ty = tid / G::NTX;
    const int x0 = blockIdx.x * TX, z = blockIdx.z;
    const int t0 = blockIdx.y * blocks_per_cta;              // first row block of this CTA
    const int nblocks = (ny + TY - 1) / TY;
    const int P = min(blocks_per_cta, nblocks - t0);          // row blocks this CTA sweeps
    const int ry0 = ty * PY;
    const int gx = x0 + 4 * tx;

    if (tid == 0) {
        ptx::prefetch_tmap(&tmap);
#pragma unroll
        for (int s = 0; s < S; ++s) ptx::mbar_init(&full[s], 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
        for (int j = 0; j < S && j < P; ++j) {
            ptx::mbar_arrive_expect_tx(&full[j], G::PLANE * sizeof(float));
            ptx::tma_load_3d(stages + j * G::STAGE, &tmap, x0, (t0 + j) * TY, z, &full[j]);
        }
    }
    __syncthreads();
    for (int j = 0; j < P; ++j) {
        const int s = j % S;
        if (tid == 0 && !ptx::mbar_wait_bounded(&full[s], (uint32_t)(j / S) & 1u, err)) abort_flag = 1;
        __syncthreads();  // block j is staged, and every thread is done with block j-1
        if (abort_flag) return;
        if (tid == 0 && j >= 1 && j - 1 + S < P) {
            const int sp = (j - 1) % S;
            ptx::mbar_arrive_expect_tx(&full[sp], G::PLANE * sizeof(float));
            ptx::tma_load_3d(stages + sp * G::STAGE, &tmap, x0, (t0 + j - 1 + S) * TY, z, &full[sp]);
        }
        float o[PY][4];
        if constexpr (BOX)
            box2d_tile<R, PY, G::BX, G::NV>(stages + s * G::STAGE, cf, o, tx, ry0);
        else
            star2d_tile<R, PY, G::BX, G::NV>(stages + s * G::STAGE, cf, o, tx, ry0);
#pragma unroll
        for (int i = 0; i < PY; ++i) {
            const int y = (t0 + j) * TY + ry0 + i;
            if (y >= ny || gx >= nx) continue;
            float *op = out + (int64_t)z * opz + (int64_t)y * opy + gx;
            if (vec_store && gx + 3 < nx) {
                *reinterpret_cast<float4 *>(op) = make_float4(o[i][0], o[i][1], o[i][2], o[i][3]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (gx + k < nx) op[k] = o[i][k];
            }
        }
    }
}

// Tile variants (TX, TY, PY, stages, row blocks per CTA).
struct PlaneVariant { int tx, ty, py, s, bpc; };
constexpr PlaneVariant kPlaneVariants[] = {
    {64, 16, 2, 3, 8}, {128, 16, 2, 3, 8}, {64, 32, 2, 3, 8},  {64, 32, 4, 3, 8},
    {128, 32, 2, 4, 16}, {64, 16, 1, 3, 16}, {128, 8, 1, 3, 16}, {64, 16, 2, 4, 32},
};
constexpr int kNumPlane = sizeof(kPlaneVariants) / sizeof(PlaneVariant);

template <int R, int TX, int TY, int PY, int S, bool BOX, typename Coef>
cudaError_t launch_plane(const Sweep &sw, const CUtensorMap &tmap, const Coef &cf, int bpc)
{
    using G = Geom<R, TX, TY, PY, S>;
    auto kern = plane_cc_kernel<R, TX, TY, PY, S, BOX, Coef>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    const int64_t nblocks = (sw.ny + TY - 1) / TY;
    const dim3 grid((unsigned)((sw.nx + TX - 1) / TX), (unsigned)((nblocks + bpc - 1) / bpc), (unsigned)sw.nz);
    const int vec = ((sw.opy % 4) == 0 && (sw.opz % 4) == 0 && (reinterpret_cast<uintptr_t>(sw.out) % 16) == 0) ? 1 : 0;
    kern<<<grid, G::NT, G::SMEM, sw.stream>>>(tmap, cf, sw.out, (int)sw.nx, (int)sw.ny, sw.opy, sw.opz, bpc, vec,
                                               device_error_word());
    return cudaGetLastError();
}

template <int R, bool BOX, typename Coef>
cudaError_t dispatch_plane(const Sweep &sw, const CUtensorMap &tmap, const Coef &cf, int v)
{
#define MMS_PLANE_CASE(I)                                                                                 \
    case I:                                                                                               \
        return launch_plane<R, kPlaneVariants[I].tx, kPlaneVariants[I].ty, kPlaneVariants[I].py,         \
                            kPlaneVariants[I].s, BOX, Coef>(sw, tmap, cf, kPlaneVariants[I].bpc);
    switch (v) {
        MMS_PLANE_CASE(0)
        MMS_PLANE_CASE(1)
        MMS_PLANE_CASE(2)
        MMS_PLANE_CASE(3)
        MMS_PLANE_CASE(4)
        MMS_PLANE_CASE(5)
        MMS_PLANE_CASE(6)
        MMS_PLANE_CASE(7)
        default: return cudaErrorInvalidValue;
    }
#undef MMS_PLANE_CASE
}

}  // namespace

int plane_cc_variants() { return kNumPlane; }

void plane_cc_box(int r, int v, int *bx, int *by)
{
    const PlaneVariant &t = kPlaneVariants[v];
    *bx = (t.tx + 2 * r + 3) & ~3;
    *by = t.ty + 2 * r;
}

cudaError_t launch_plane_cc(const Sweep &s, const CUtensorMap &tmap, int v)
{
    const int w = 2 * s.r + 1;
    if (s.shape == MMS_BOX2D) {
        BoxCoef cf{};
        for (int i = 0; i < w * w; ++i) cf.c[i] = s.coeffs[i];
        switch (s.r) {
            case 1: return dispatch_plane<1, true>(s, tmap, cf, v);
            case 2: return dispatch_plane<2, true>(s, tmap, cf, v);
            case 3: return dispatch_plane<3, true>(s, tmap, cf, v);
            case 4: return dispatch_plane<4, true>(s, tmap, cf, v);
            default: return cudaErrorInvalidValue;
        }
    }
    StarCoef cf{};
    for (int i = 0; i < 2 * w; ++i) cf.c[i] = s.coeffs[i];
    switch (s.r) {
        case 1: return dispatch_plane<1, false>(s, tmap, cf, v);
        case 2: return dispatch_plane<2, false>(s, tmap, cf, v);
        case 3: return dispatch_plane<3, false>(s, tmap, cf, v);
        case 4: return dispatch_plane<4, false>(s, tmap, cf, v);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mms
