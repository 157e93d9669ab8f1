// tile.cuh -- the shared-memory plane tile of the CUDA-core sweeps and of
// the fused wave kernels: its geometry and the per-plane star and box
// updates of a thread's register queue of partial sums.
#pragma once

#include "common.cuh"

namespace mms {

// The dynamic shared-memory base rounded up to 128 bytes (TMA destinations
// need 128-byte alignment; the launch adds 128 bytes of slack for this).
__device__ __forceinline__ unsigned char *smem_align128(unsigned char *p)
{
    const uint32_t a = ptx::smem_u32(p);  // offset in the shared window
    return p + ((128u - (a & 127u)) & 127u);
}

template <int R, int TX, int TY, int PY, int S>
struct Geom {
    static constexpr int W = 2 * R + 1;
    static constexpr int BX = (TX + 2 * R + 3) & ~3;  // TMA box x: a 16-byte multiple
    static constexpr int BY = TY + 2 * R;
    static constexpr int PLANE = BX * BY;             // floats one TMA box writes
    static constexpr int STAGE = (PLANE + 31) & ~31;  // ring stride: 128-byte multiple
    static constexpr int NTX = TX / 4;                // threads along x (4 points each)
    static constexpr int NT = NTX * (TY / PY);
    static constexpr int NV = (4 + 2 * R + 3) / 4;    // float4 per window row
    // 128 bytes of slack to align the dynamic base, the ring, its barriers
    // and the CTA's abort flag.
    static constexpr size_t SMEM = 128 + (size_t)S * STAGE * sizeof(float) + S * sizeof(uint64_t) + 16;
    static_assert(TX % 4 == 0 && TY % PY == 0, "tile");
    static_assert(BX <= 256 && BY <= 256, "TMA box dims are at most 256");
    static_assert(4 * (NTX - 1) + 4 * NV <= BX, "window inside the staged row");
};

// Loads the NV float4 of a window row starting at `p` (16-byte aligned).
template <int NV>
__device__ __forceinline__ void load_row(const float *p, float (&v)[4 * NV])
{
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const float4 t = *reinterpret_cast<const float4 *>(p + 4 * q);
        v[4 * q + 0] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
}

// The 4 values at columns R..R+3 of a row whose column 0 is 16-byte aligned.
template <int R>
__device__ __forceinline__ void load_center(const float *p, float (&v)[4])
{
    constexpr int A = (R / 4) * 4;
    constexpr int o = R - A;
    const float4 t0 = *reinterpret_cast<const float4 *>(p + A);
    if constexpr (o == 0) {
        v[0] = t0.x; v[1] = t0.y; v[2] = t0.z; v[3] = t0.w;
    } else {
        const float4 t1 = *reinterpret_cast<const float4 *>(p + A + 4);
        const float tmp[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = tmp[o + k];
    }
}

// Queue slots: logical slot kk (output plane j - 2R + kk for input plane j)
// lives in acc[(kk + ROT) % (2R+1)]; ROT = 0 for a queue that is shifted
// after every plane, a compile-time rotation for one that is not.
//
// Star: plane j adds c_z[R-kk] * centre to the output plane at queue slot kk
// and its in-plane x/y part to slot R (the plane it centres); the centre
// values of the thread's points are returned in ctr.
template <int R, int PY, int BX, int NV, int ROT = 0>
__device__ __forceinline__ void star_plane(const float *pl, const StarCoef &cf,
                                           float (&acc)[2 * R + 1][PY][4], float (&ctr)[PY][4],
                                           int tx, int ry0)
{
    constexpr int W = 2 * R + 1;
    float cen[PY + 2 * R][4];
#pragma unroll
    for (int rr = 0; rr < PY + 2 * R; ++rr) load_center<R>(pl + (ry0 + rr) * BX + 4 * tx, cen[rr]);
#pragma unroll
    for (int i = 0; i < PY; ++i) {
        float win[4 * NV];
        load_row<NV>(pl + (ry0 + R + i) * BX + 4 * tx, win);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float c0 = cen[i + R][k];
            ctr[i][k] = c0;
            float xy = 0.f;
#pragma unroll
            for (int d = -R; d <= R; ++d) xy = fmaf(cf.c[0 * W + d + R], win[k + R + d], xy);
#pragma unroll
            for (int d = -R; d <= R; ++d) xy = fmaf(cf.c[1 * W + d + R], cen[i + R + d][k], xy);
            acc[(R + ROT) % W][i][k] += xy;
#pragma unroll
            for (int kk = 0; kk < W; ++kk)
                acc[(kk + ROT) % W][i][k] = fmaf(cf.c[2 * W + 2 * R - kk], c0, acc[(kk + ROT) % W][i][k]);
        }
    }
}

// Box: window row rr of the plane feeds output row i with dy = rr - R - i;
// slot kk (output plane z_o) takes the weights of dz = R - kk.
template <int R, int PY, int BX, int NV, int ROT = 0>
__device__ __forceinline__ void box_plane(const float *pl, const BoxCoef &cf,
                                          float (&acc)[2 * R + 1][PY][4], int tx, int ry0)
{
    constexpr int W = 2 * R + 1;
#pragma unroll
    for (int rr = 0; rr < PY + 2 * R; ++rr) {
        float row[4 * NV];
        load_row<NV>(pl + (ry0 + rr) * BX + 4 * tx, row);
#pragma unroll
        for (int i = 0; i < PY; ++i) {
            const int dy = rr - R - i;
            if (dy < -R || dy > R) continue;
#pragma unroll
            for (int kk = 0; kk < W; ++kk) {
                const int dz = R - kk;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float a = acc[(kk + ROT) % W][i][k];
#pragma unroll
                    for (int dx = -R; dx <= R; ++dx)
                        a = fmaf(cf.c[((dz + R) * W + dy + R) * W + dx + R], row[k + R + dx], a);
                    acc[(kk + ROT) % W][i][k] = a;
                }
            }
        }
    }
}

// Planar star (Table I's 2D kernels): the thread's 4 x PY outputs of a staged
// tile, x line (weights c[0..2R]) plus y line (weights c[2R+1..4R+1]).
template <int R, int PY, int BX, int NV>
__device__ __forceinline__ void star2d_tile(const float *pl, const StarCoef &cf, float (&o)[PY][4], int tx,
                                            int ry0)
{
    constexpr int W = 2 * R + 1;
    float cen[PY + 2 * R][4];
#pragma unroll
    for (int rr = 0; rr < PY + 2 * R; ++rr) load_center<R>(pl + (ry0 + rr) * BX + 4 * tx, cen[rr]);
#pragma unroll
    for (int i = 0; i < PY; ++i) {
        float win[4 * NV];
        load_row<NV>(pl + (ry0 + R + i) * BX + 4 * tx, win);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float acc = 0.f;
#pragma unroll
            for (int d = -R; d <= R; ++d) acc = fmaf(cf.c[d + R], win[k + R + d], acc);
#pragma unroll
            for (int d = -R; d <= R; ++d) acc = fmaf(cf.c[W + d + R], cen[i + R + d][k], acc);
            o[i][k] = acc;
        }
    }
}

// Planar box: window row rr of the tile feeds output row i with dy = rr - R - i.
template <int R, int PY, int BX, int NV>
__device__ __forceinline__ void box2d_tile(const float *pl, const BoxCoef &cf, float (&o)[PY][4], int tx,
                                           int ry0)
{
    constexpr int W = 2 * R + 1;
#pragma unroll
    for (int i = 0; i < PY; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) o[i][k] = 0.f;
#pragma unroll
    for (int rr = 0; rr < PY + 2 * R; ++rr) {
        float row[4 * NV];
        load_row<NV>(pl + (ry0 + rr) * BX + 4 * tx, row);
#pragma unroll
        for (int i = 0; i < PY; ++i) {
            const int dy = rr - R - i;
            if (dy < -R || dy > R) continue;
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int dx = -R; dx <= R; ++dx)
                    o[i][k] = fmaf(cf.c[(dy + R) * W + dx + R], row[k + R + dx], o[i][k]);
        }
    }
}

}  // namespace mms
