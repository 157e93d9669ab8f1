// sweep_cc.cuh -- the FP32 CUDA-core sweep kernel shared by the star
// (sweep_star.cu) and box (sweep_cc.cu) translation units: one TMA plane
// ring per CTA, a register queue of 2R+1 partial sums per point along z,
// float4 stores.  See sweep_cc.cu for the design.
#pragma once

#include <utility>

#include "common.cuh"
#include "tile.cuh"

namespace mms {
namespace sweep {

// Tile variant: TX x TY outputs per CTA, PY rows per thread, S ring stages,
// TZ planes per CTA, rotated (true) or shifted (false) queue, and whether one
// thread waits for each staged plane while the others block at the CTA
// barrier (true) or every thread polls the stage's mbarrier (false).
struct Variant { int tx, ty, py, s, tz; bool rot; bool one_wait = false; };

// Box tile variants (shared by the radius-1/2 and radius-3/4 units).
constexpr Variant kBoxVariants[] = {
    {64, 16, 2, 3, 64, false},  {64, 32, 2, 3, 64, false},  {32, 16, 2, 3, 64, false},
    {64, 16, 4, 3, 64, false},  {64, 8, 2, 3, 128, false},  {128, 16, 2, 3, 32, false},
    {64, 16, 1, 3, 128, false}, {64, 8, 1, 3, 128, false},  {128, 16, 2, 3, 32, true},
    {64, 16, 2, 3, 64, true},   {128, 16, 2, 3, 32, true, true}, {64, 8, 2, 3, 128, false, true},
};
constexpr int kNumBox = sizeof(kBoxVariants) / sizeof(Variant);

// The box sweep of radius 3 or 4 (sweep_box_high.cu).
cudaError_t launch_box_cc_high(const Sweep &s, const CUtensorMap &tmap, const BoxCoef &cf, int v);

// One plane step of a sweep: wait for plane j, add it to the queue, hand
// the stage back to TMA, store the output plane it completes and free its
// slot.  ROT = -1: the queue is shifted after the plane (slot 0 is the
// oldest); ROT >= 0: the queue is rotated instead, the oldest partial sum in
// slot ROT (the caller unrolls 2R+1 planes so ROT is a constant).  ONEW: one
// thread waits for the stage and the CTA barrier releases the others (and
// tells thread 0 that plane j-1's stage is free); otherwise every thread
// polls the mbarrier and the barrier follows the plane.  Returns false when
// the CTA aborts (a bounded wait ran out).
template <int R, int TX, int TY, int PY, int S, bool BOX, int ROT, bool ONEW, typename Coef>
__device__ __forceinline__ bool plane_step(int j, int P, const CUtensorMap &tmap, const Coef &cf,
                                           float *planes, uint64_t *full, int &abort_flag,
                                           float (&acc)[2 * R + 1][PY][4], float *out, int nx, int ny,
                                           int64_t opy, int64_t opz, int x0, int y0, int zb, int tx,
                                           int ry0, int gx, int vec_store, unsigned *err)
{
    using G = Geom<R, TX, TY, PY, S>;
    constexpr int W = G::W;
    constexpr int Q = ROT < 0 ? 0 : ROT;  // physical slot of the oldest partial sum
    const int s = j % S;
    if constexpr (ONEW) {
        if (threadIdx.x == 0 && !ptx::mbar_wait_bounded(&full[s], (uint32_t)(j / S) & 1u, err)) abort_flag = 1;
        __syncthreads();  // stage s is full for all, and every thread is done with plane j-1
        if (abort_flag) return false;
        if (threadIdx.x == 0 && j >= 1 && j - 1 + S < P) {
            const int sp = (j - 1) % S;
            ptx::mbar_arrive_expect_tx(&full[sp], G::PLANE * sizeof(float));
            ptx::tma_load_3d(planes + sp * G::STAGE, &tmap, x0, y0, zb + j - 1 + S, &full[sp]);
        }
        const float *pl = planes + s * G::STAGE;
        if constexpr (BOX)
            box_plane<R, PY, G::BX, G::NV, Q>(pl, cf, acc, tx, ry0);
        else {
            float ctr[PY][4];
            star_plane<R, PY, G::BX, G::NV, Q>(pl, cf, acc, ctr, tx, ry0);
        }
    } else {
        if (ptx::mbar_wait_bounded(&full[s], (uint32_t)(j / S) & 1u, err)) {
            const float *pl = planes + s * G::STAGE;
            if constexpr (BOX)
                box_plane<R, PY, G::BX, G::NV, Q>(pl, cf, acc, tx, ry0);
            else {
                float ctr[PY][4];
                star_plane<R, PY, G::BX, G::NV, Q>(pl, cf, acc, ctr, tx, ry0);
            }
        } else {
            abort_flag = 1;
        }
        __syncthreads();  // every thread is done with stage s
        if (abort_flag) return false;
        if (threadIdx.x == 0 && j + S < P) {
            ptx::mbar_arrive_expect_tx(&full[s], G::PLANE * sizeof(float));
            ptx::tma_load_3d(planes + s * G::STAGE, &tmap, x0, y0, zb + j + S, &full[s]);
        }
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
                        make_float4(acc[Q][i][0], acc[Q][i][1], acc[Q][i][2], acc[Q][i][3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (gx + k < nx) o[k] = acc[Q][i][k];
                }
            }
        }
    }
    if constexpr (ROT < 0) {
#pragma unroll
        for (int kk = 0; kk < W - 1; ++kk)
#pragma unroll
            for (int i = 0; i < PY; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[kk][i][k] = acc[kk + 1][i][k];
    }
    // the freed slot becomes the newest output plane's
    constexpr int FREE = ROT < 0 ? W - 1 : Q;
#pragma unroll
    for (int i = 0; i < PY; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[FREE][i][k] = 0.f;
    return true;
}

// Runs planes j0 .. j0+2R (those below P) with the queue rotated: input
// plane j = j0 + u keeps its oldest partial sum (output plane j - 2R) in
// slot (u + 1) mod (2R+1).
template <int R, int TX, int TY, int PY, int S, bool BOX, bool ONEW, typename Coef, int... U>
__device__ __forceinline__ bool rotated_block(std::integer_sequence<int, U...>, int j0, int P,
                                              const CUtensorMap &tmap, const Coef &cf, float *planes,
                                              uint64_t *full, int &abort_flag,
                                              float (&acc)[2 * R + 1][PY][4], float *out, int nx, int ny,
                                              int64_t opy, int64_t opz, int x0, int y0, int zb, int tx,
                                              int ry0, int gx, int vec_store, unsigned *err)
{
    bool ok = true;
    ((ok = ok && (j0 + U >= P ||
                  plane_step<R, TX, TY, PY, S, BOX, (U + 1) % (2 * R + 1), ONEW>(
                      j0 + U, P, tmap, cf, planes, full, abort_flag, acc, out, nx, ny, opy, opz, x0, y0,
                      zb, tx, ry0, gx, vec_store, err))),
     ...);
    return ok;
}

template <int R, int TX, int TY, int PY, int S, bool BOX, bool ROTQ, bool ONEW, typename Coef>
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

    // The box rotates only for R <= 2: above that its 2R+1 unrolled copies
    // of a (2R+1)^3-term plane update cost more than the moves they save.
    constexpr bool ROTATE = ROTQ && (!BOX || R <= 2);
    if constexpr (ROTATE) {
        // 2R+1 planes per iteration, so every queue slot index is a constant
        // and no partial sum is moved between registers
        for (int j0 = 0; j0 < P; j0 += W)
            if (!rotated_block<R, TX, TY, PY, S, BOX, ONEW, Coef>(std::make_integer_sequence<int, W>{}, j0, P,
                                                            tmap, cf, planes, full, abort_flag, acc, out,
                                                            nx, ny, opy, opz, x0, y0, zb, tx, ry0, gx,
                                                            vec_store, err))
                return;
    } else {
        for (int j = 0; j < P; ++j)
            if (!plane_step<R, TX, TY, PY, S, BOX, -1, ONEW>(j, P, tmap, cf, planes, full, abort_flag, acc, out,
                                                       nx, ny, opy, opz, x0, y0, zb, tx, ry0, gx,
                                                       vec_store, err))
                return;
    }
}

template <int R, int TX, int TY, int PY, int S, bool BOX, bool ROTQ, bool ONEW, typename Coef>
cudaError_t launch_tiled(const Sweep &sw, const CUtensorMap &tmap, const Coef &cf, int tz)
{
    using G = Geom<R, TX, TY, PY, S>;
    auto kern = sweep_cc_kernel<R, TX, TY, PY, S, BOX, ROTQ, ONEW, Coef>;
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

// Runs variant v of table TAB (a constexpr array of Variant).
#define MMS_SWEEP_DISPATCH(TAB, R, BOX, Coef, sw, tmap, cf, v)                                  \
    switch (v) {                                                                                \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 0)                                      \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 1)                                      \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 2)                                      \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 3)                                      \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 4)                                      \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 5)                                      \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 6)                                      \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 7)                                      \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 8)                                      \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 9)                                      \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 10)                                     \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 11)                                     \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 12)                                     \
        MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, 13)                                     \
        default: return cudaErrorInvalidValue;                                                  \
    }
#define MMS_SWEEP_CASE(TAB, R, BOX, Coef, sw, tmap, cf, I)                                      \
    case I:                                                                                     \
        if constexpr (I < (int)(sizeof(TAB) / sizeof(Variant)))                                 \
            return launch_tiled<R, TAB[I].tx, TAB[I].ty, TAB[I].py, TAB[I].s, BOX, TAB[I].rot,        \
                                TAB[I].one_wait, Coef>(                                           \
                sw, tmap, cf, TAB[I].tz);                                                       \
        else                                                                                    \
            return cudaErrorInvalidValue;

}  // namespace sweep
}  // namespace mms
