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

#include "sweep_cc.cuh"

namespace mms {
namespace {

using sweep::Variant;
using sweep::launch_tiled;

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
        // the planar shapes have no z halo
        const float *c0 = in + (z + (is_planar(shape) ? 0 : r)) * ipz + (y + r) * ipy + (x + r);
        float acc = 0.f;
        if (shape == MMS_STAR2D) {
            for (int d = -r; d <= r; ++d) {
                acc = fmaf(cf.c[d + r], c0[d], acc);
                acc = fmaf(cf.c[w + d + r], c0[d * ipy], acc);
            }
        } else if (shape == MMS_BOX2D) {
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx)
                    acc = fmaf(cf.c[(dy + r) * w + dx + r], c0[dy * ipy + dx], acc);
        } else if (shape == MMS_STAR) {
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

using sweep::kBoxVariants;

template <int R>
cudaError_t dispatch_box(const Sweep &sw, const CUtensorMap &tmap, const BoxCoef &cf, int v)
{
    MMS_SWEEP_DISPATCH(kBoxVariants, R, true, BoxCoef, sw, tmap, cf, v)
}

}  // namespace

int box_cc_variants() { return sweep::kNumBox; }

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
    const int n = s.shape == MMS_STAR ? 3 * w : s.shape == MMS_BOX ? w * w * w : s.shape == MMS_STAR2D ? 2 * w : w * w;
    for (int i = 0; i < n; ++i) cf.c[i] = s.coeffs[i];
    const int64_t total = s.nx * s.ny * s.nz;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    naive_kernel<<<blocks, 256, 0, s.stream>>>(s.shape, s.r, cf, s.in, s.ipy, s.ipz, s.out, s.opy,
                                              s.opz, s.nx, s.ny, s.nz);
    return cudaGetLastError();
}

cudaError_t launch_box_cc(const Sweep &s, const CUtensorMap &tmap, int v)
{
    BoxCoef cf{};
    const int w = 2 * s.r + 1;
    for (int i = 0; i < w * w * w; ++i) cf.c[i] = s.coeffs[i];
    switch (s.r) {
        case 1: return dispatch_box<1>(s, tmap, cf, v);
        case 2: return dispatch_box<2>(s, tmap, cf, v);
        case 3:
        case 4: return sweep::launch_box_cc_high(s, tmap, cf, v);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mms
