// sweep_f64.cu -- FP64 star and box sweeps (3D and the planar 2D shapes).
//
// GB300's FP64 pipe issues about two FMAs per clock per SM, 1/64 of the
// FP32 rate, so an FP64 sweep is bound by that pipe long before HBM (star
// r = 4: 25 FMAs per 16 bytes moved).  The kernel therefore spends nothing
// on staging: one thread per output point, neighbours through the read-only
// L1 path (each input is reused from L1/L2 by the threads around it), and
// the FMA count cut to the minimum -- the star's three centre weights are
// folded into one, so a radius-r star costs 6r + 1 FMAs and a box (2r+1)^3.
#include "common.cuh"

namespace mms {

namespace {

struct F64Coef { double c[(2 * kMaxR + 1) * (2 * kMaxR + 1) * (2 * kMaxR + 1)]; };

template <int SHAPE, int R>
__global__ void __launch_bounds__(256)
    f64_kernel(const __grid_constant__ F64Coef cf, const double *__restrict__ in, int64_t ipy, int64_t ipz,
               double *__restrict__ out, int64_t opy, int64_t opz, int nx, int ny, int nz)
{
    constexpr int W = 2 * R + 1;
    const int x = blockIdx.x * 32 + threadIdx.x;
    if (x >= nx) return;
    constexpr bool planar = SHAPE == MMS_STAR2D || SHAPE == MMS_BOX2D;
    // y and z stride over the grid's extents (launch dims are capped at 65535)
    for (int z = blockIdx.z; z < nz; z += gridDim.z)
        for (int y = blockIdx.y * 8 + threadIdx.y; y < ny; y += gridDim.y * 8) {
            const double *c0 = in + (int64_t)(z + (planar ? 0 : R)) * ipz + (int64_t)(y + R) * ipy + (x + R);
            double acc;
            if constexpr (SHAPE == MMS_STAR || SHAPE == MMS_STAR2D) {
                constexpr int NA = SHAPE == MMS_STAR ? 3 : 2;
                double cc = cf.c[R] + cf.c[W + R];
                if constexpr (NA == 3) cc += cf.c[2 * W + R];
                acc = cc * __ldg(c0);
#pragma unroll
                for (int d = 1; d <= R; ++d) {
                    acc = fma(cf.c[R + d], __ldg(c0 + d), acc);
                    acc = fma(cf.c[R - d], __ldg(c0 - d), acc);
                    acc = fma(cf.c[W + R + d], __ldg(c0 + d * ipy), acc);
                    acc = fma(cf.c[W + R - d], __ldg(c0 - d * ipy), acc);
                    if constexpr (NA == 3) {
                        acc = fma(cf.c[2 * W + R + d], __ldg(c0 + d * ipz), acc);
                        acc = fma(cf.c[2 * W + R - d], __ldg(c0 - d * ipz), acc);
                    }
                }
            } else if constexpr (SHAPE == MMS_BOX2D) {
                acc = 0.0;
#pragma unroll
                for (int dy = -R; dy <= R; ++dy)
#pragma unroll
                    for (int dx = -R; dx <= R; ++dx)
                        acc = fma(cf.c[(dy + R) * W + dx + R], __ldg(c0 + dy * ipy + dx), acc);
            } else {
                acc = 0.0;
#pragma unroll 1
                for (int dz = -R; dz <= R; ++dz)
#pragma unroll
                    for (int dy = -R; dy <= R; ++dy)
#pragma unroll
                        for (int dx = -R; dx <= R; ++dx)
                            acc = fma(cf.c[((dz + R) * W + dy + R) * W + dx + R], __ldg(c0 + dz * ipz + dy * ipy + dx), acc);
            }
            out[(int64_t)z * opz + (int64_t)y * opy + x] = acc;
        }
}

template <int SHAPE>
cudaError_t f64_shape(int r, const F64Coef &cf, const double *in, int64_t ipy, int64_t ipz, double *out,
                      int64_t opy, int64_t opz, int nx, int ny, int nz, cudaStream_t st)
{
    const dim3 block(32, 8), grid((nx + 31) / 32, min((ny + 7) / 8, 65535), min(nz, 65535));
    switch (r) {
        case 1: f64_kernel<SHAPE, 1><<<grid, block, 0, st>>>(cf, in, ipy, ipz, out, opy, opz, nx, ny, nz); break;
        case 2: f64_kernel<SHAPE, 2><<<grid, block, 0, st>>>(cf, in, ipy, ipz, out, opy, opz, nx, ny, nz); break;
        case 3: f64_kernel<SHAPE, 3><<<grid, block, 0, st>>>(cf, in, ipy, ipz, out, opy, opz, nx, ny, nz); break;
        case 4: f64_kernel<SHAPE, 4><<<grid, block, 0, st>>>(cf, in, ipy, ipz, out, opy, opz, nx, ny, nz); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_f64(int shape, int r, const double *coeffs, int ncoef, const double *in, int64_t ipy, int64_t ipz,
                       double *out, int64_t opy, int64_t opz, int64_t nx, int64_t ny, int64_t nz, cudaStream_t st)
{
    F64Coef cf{};
    for (int i = 0; i < ncoef; ++i) cf.c[i] = coeffs[i];
    const int X = (int)nx, Y = (int)ny, Z = (int)nz;
    switch (shape) {
        case MMS_STAR: return f64_shape<MMS_STAR>(r, cf, in, ipy, ipz, out, opy, opz, X, Y, Z, st);
        case MMS_BOX: return f64_shape<MMS_BOX>(r, cf, in, ipy, ipz, out, opy, opz, X, Y, Z, st);
        case MMS_STAR2D: return f64_shape<MMS_STAR2D>(r, cf, in, ipy, ipz, out, opy, opz, X, Y, Z, st);
        case MMS_BOX2D: return f64_shape<MMS_BOX2D>(r, cf, in, ipy, ipz, out, opy, opz, X, Y, Z, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mms
