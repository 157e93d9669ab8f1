// common.cuh -- shared internals of the sm_103a stencil library: launch
// argument structs, the device error word, and inline-PTX helpers for
// mbarriers, TMA bulk-tensor copies and the global timer.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mms.h"

namespace mms {

// Largest radius and coefficient counts (star: 3*(2r+1), box: (2r+1)^3).
constexpr int kMaxR = 4;
constexpr int kMaxStar = 3 * (2 * kMaxR + 1);
constexpr int kMaxBox = (2 * kMaxR + 1) * (2 * kMaxR + 1) * (2 * kMaxR + 1);

// Coefficients travel as kernel parameters (constant bank), so every FMA
// reads its weight as a uniform constant operand.
struct StarCoef { float c[kMaxStar]; };
struct BoxCoef { float c[kMaxBox]; };

// Device error word bits (read by mms_check_device).
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned kErrIndex = 2u;

// Bound of every device-side wait (nanoseconds of %globaltimer).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// One sweep, as validated by the ABI layer.
struct Sweep {
    int shape, r;
    int64_t nx, ny, nz;
    const float *in;
    int64_t ipy, ipz;
    float *out;
    int64_t opy, opz;
    const float *coeffs;  // host
    int variant;
    cudaStream_t stream;
};

// Host launchers (each returns a CUDA error code; validation happens above).
cudaError_t launch_naive(const Sweep &s);
cudaError_t launch_star_cc(const Sweep &s, const CUtensorMap &tmap, int variant);
cudaError_t launch_box_cc(const Sweep &s, const CUtensorMap &tmap, int variant);
int star_cc_variants();
int box_cc_variants();
// TMA box (x extent, y extent) that variant v of the CUDA-core sweeps loads.
void star_cc_box(int r, int v, int *bx, int *by);
void box_cc_box(int r, int v, int *bx, int *by);

// Planar (2D) CUDA-core sweeps (sweep_2d.cu).
cudaError_t launch_plane_cc(const Sweep &s, const CUtensorMap &tmap, int variant);
int plane_cc_variants();
void plane_cc_box(int r, int v, int *bx, int *by);

// Planar shapes have no z halo.
__host__ __device__ constexpr bool is_planar(int shape) { return shape == MMS_STAR2D || shape == MMS_BOX2D; }

// Tensor-core banded sweeps (band_tc.cu).
int band_tc_supported(int shape, int r, int path);
// The star's two-pass variants run a planar tensor-core pass into `scratch`
// (nx*ny*nz floats, dense; band_tc_scratch_bytes of the sweep with its
// resolved variant in Sweep::variant) followed by a CUDA-core z pass; every
// other variant needs no scratch.
cudaError_t launch_band_tc(const Sweep &s, int path, const CUtensorMap &tmap, int variant, float *scratch);
size_t band_tc_scratch_bytes(const Sweep &s);
void band_tc_box(int shape, int r, int path, int v, int *bx, int *by, int *bz, int *swz);
int band_tc_variants(int shape, int r, int path);

// Error word helpers (wave.cu owns the symbol).
unsigned *device_error_word();

// Encodes a 3D FP32 tensor map over a padded grid (x extent X, pitches in
// elements) with box (bx, by, bz); returns false when the driver refuses.
bool encode_tmap_3d(CUtensorMap *map, const float *base, int64_t X, int64_t Y, int64_t Z,
                    int64_t py, int64_t pz, int bx, int by, int bz, bool swizzle128 = false);
// The same over nw stacked grids `pw` elements apart, box depth 1 in w.
bool encode_tmap_4d(CUtensorMap *map, const float *base, int64_t X, int64_t Y, int64_t Z,
                    int64_t W, int64_t py, int64_t pz, int64_t pw, int bx, int by, int bz);

}  // namespace mms

// ------------------------------------------------------------ PTX helpers
namespace ptx {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// One lane of the (converged, full) warp is elected; true in that lane.
__device__ __forceinline__ bool elect_one()
{
    uint32_t pred = 0;
    asm volatile("{\n\t.reg .pred p;\n\telect.sync _|p, 0xffffffff;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(pred));
    return pred != 0;
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete; gives up after
// limit_ns (kWaitLimitNs by default), sets the timeout bit of the device
// error word and returns false.  Never traps.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned *err,
                                                  unsigned long long limit_ns = mms::kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u && globaltimer() - t0 > limit_ns) {
            if (err) atomicOr(err, mms::kErrTimeout);
            return false;
        }
    }
}

// TMA: 3D tiled load global -> shared, completion counted on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// TMA: 4D tiled load global -> shared (x, y, z, w coordinates).
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            int w, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

}  // namespace ptx
