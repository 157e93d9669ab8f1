// band_tc.cu -- box stencil sweeps on the tcgen05 tensor cores.
//
// The paper (Sec. 4.1) turns a 1D stencil into an outer-product / matrix
// product with a banded coefficient matrix, and (Sec. 4.3) a box stencil
// into 2r+1 shifted 1D stencils.  On GB300 the contraction runs on tcgen05
// MMAs, arranged so that the banded operand is small and sits in tensor
// memory and the data operand is the wide one:
//
//   D[(dy, x), line] += sum_k  Band_dz[(dy, x), k] * Data[k, line + dz*YP]
//
//  * M = 128 TMEM lanes hold (dy, x) pairs: 2r+1 row offsets dy times TXO
//    output x positions; Band_dz[(dy, x), k] = c[dz][dy][k - x] (zero off
//    the band), split into hi/lo parts, written to TMEM once per CTA;
//  * K runs over TXO + 2r input x positions (the band width);
//  * N = lines: NZ output planes x YP staged rows.  The data operand is the
//    staged input converted to BF16 (or TF32) hi/lo parts in the K-major
//    canonical layout; the dz shift of the box is a start-address offset of
//    its shared-memory descriptor (whole planes), so the 2r+1 planes of the
//    box accumulate into one TMEM accumulator without moving data;
//  * the remaining sum over dy (2r+1 lanes, rows shifted by dy) happens in
//    the epilogue: TMEM -> registers -> shared memory -> FP32 adds -> global.
// Split precision (3 products hi*hi + hi*lo + lo*hi, FP32 accumulation)
// recovers FP32-level accuracy from BF16 or TF32 operands.
//
// Pipeline (persistent CTAs, one per SM, 128 threads): TMA stages the FP32
// box of group i+2 while group i is converted and its MMAs run; the
// epilogue of group i-1 drains the other TMEM accumulator meanwhile.
#include <cuda_bf16.h>
#include <stdio.h>

#include "common.cuh"
#include "tc.cuh"

namespace mms {
namespace {

enum { P_TF32 = 0, P_3XTF32 = 1, P_BF16X3 = 2 };

constexpr int roundup(int a, int b) { return (a + b - 1) / b * b; }

template <int R, int PREC>
struct Cfg {
    static constexpr bool BF = PREC == P_BF16X3;
    static constexpr int ELT = BF ? 2 : 4;           // operand bytes
    static constexpr int KSTEP = BF ? 16 : 8;        // K of one MMA instruction
    static constexpr int KC = 16 / ELT;              // K elements per 16-byte chunk
    static constexpr int W = 2 * R + 1;
    static constexpr int TXO = R == 1 ? 40 : R == 2 ? 24 : R == 3 ? 16 : 12;  // x outputs per tile
    static constexpr int LANES = W * TXO;            // used TMEM lanes (<= 128)
    static constexpr int K = roundup(TXO + 2 * R, KSTEP);
    static constexpr int NPARTS = PREC == P_TF32 ? 1 : 2;
    static constexpr int NPROD = PREC == P_TF32 ? 1 : 3;
    static constexpr int BANDCOLS = K * ELT / 4;     // 32-bit TMEM columns per band part
    static constexpr int BAND_TOTAL = W * NPARTS * BANDCOLS;
    static constexpr int YP = 32;                    // staged rows per plane
    static constexpr int TY = YP - 2 * R;            // output rows per tile
    static constexpr int NZ = (2 * 4 * YP + BAND_TOTAL <= 512)   ? 4
                              : (2 * 3 * YP + BAND_TOTAL <= 512) ? 3
                              : (2 * 2 * YP + BAND_TOTAL <= 512) ? 2
                                                                 : 1;
    static constexpr bool OK = 2 * NZ * YP + BAND_TOTAL <= 512 && LANES <= 128;
    static constexpr int N = NZ * YP;                // MMA N (lines per group)
    static constexpr int ZS = NZ + 2 * R;            // staged planes per group
    static constexpr int NL = ZS * YP;               // staged lines per group
    static constexpr int STG_BYTES = NL * K * 4;     // FP32 TMA staging
    static constexpr int PART_BYTES = NL * K * ELT;  // one converted operand part
    static constexpr int CONV_BYTES = PART_BYTES * NPARTS;
    static constexpr int DSM_LD = 33;                // epilogue row stride (floats)
    static constexpr int DSM_BYTES = 128 * DSM_LD * 4;
    static constexpr int NT = 128;
    static constexpr int BAND_COL0 = 2 * N;          // TMEM: D0 | D1 | bands
    static constexpr uint32_t IDESC = tc::instr_desc(BF ? 1u : 2u, 128, N);
    // shared memory: [stg0 stg1 | conv0 conv1 | dsm | barriers, tmem slot, flag]
    static constexpr size_t OFF_CONV = 2 * (size_t)STG_BYTES;
    static constexpr size_t OFF_DSM = OFF_CONV + 2 * (size_t)CONV_BYTES;
    static constexpr size_t OFF_BAR = OFF_DSM + DSM_BYTES;
    static constexpr size_t SMEM = 128 + OFF_BAR + 64;
    static_assert(N % 16 == 0 && N <= 256, "MMA N");
    static_assert(STG_BYTES % 128 == 0 && CONV_BYTES % 128 == 0 && PART_BYTES % 16 == 0, "align");
};

__device__ __forceinline__ uint32_t bf16_bits(float v)
{
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
}

__device__ __forceinline__ float bf16_val(uint32_t b)
{
    return __bfloat162float(__ushort_as_bfloat16((unsigned short)b));
}

__device__ __forceinline__ uint32_t tf32_rna(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

// hi/lo split of one value for operand part p (0 = hi, 1 = lo), as raw bits
// of the operand type.
template <int PREC>
__device__ __forceinline__ uint32_t split_part(float v, int p)
{
    if constexpr (PREC == P_BF16X3) {
        const uint32_t h = bf16_bits(v);
        return p == 0 ? h : bf16_bits(v - bf16_val(h));
    } else {
        const uint32_t h = tf32_rna(v);
        return p == 0 ? h : tf32_rna(v - __uint_as_float(h));
    }
}

struct TcArgs {
    float *out;
    int64_t opy, opz;
    int nx, ny, nz;
    int tiles_x, tiles_y, tiles;  // tiles = tiles_x * tiles_y * zchunks
    int groups;                   // groups (of NZ planes) per tile
};

template <int R, int PREC>
__global__ void __launch_bounds__(128, 1)
    box_tc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ BoxCoef cf,
                  const __grid_constant__ TcArgs a, unsigned *err)
{
    using C = Cfg<R, PREC>;
    constexpr int W = C::W;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (ptx::smem_u32(smem_raw) & 127u)) & 127u);
    float *stg = reinterpret_cast<float *>(smem);
    unsigned char *conv = smem + C::OFF_CONV;
    float *dsm = reinterpret_cast<float *>(smem + C::OFF_DSM);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);  // [2]
    uint64_t *mmad = full + 2;                                         // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mmad + 2);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int my_tiles = a.tiles > (int)blockIdx.x ? (a.tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int ng = my_tiles * a.groups;

    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&full[b], 1);
            ptx::mbar_init(&mmad[b], 1);
        }
        ptx::fence_mbar_init();
        *abort_flag = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tmem_slot;

    // Banded coefficient operand: lane (dy, x) of part p for plane offset dz.
    {
        const int l = warp * 32 + lane;
        const bool used = l < C::LANES;
        const int dyi = used ? l / C::TXO : 0, xo = used ? l % C::TXO : 0;
        for (int dzi = 0; dzi < W; ++dzi)
            for (int p = 0; p < C::NPARTS; ++p)
                for (int c0 = 0; c0 < C::BANDCOLS; c0 += 8) {
                    uint32_t v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        uint32_t word = 0;
                        if constexpr (C::BF) {
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int k = 2 * (c0 + j) + h, d = k - xo;
                                uint32_t bits = 0;
                                if (used && d >= 0 && d <= 2 * R)
                                    bits = split_part<PREC>(cf.c[(dzi * W + dyi) * W + d], p);
                                word |= bits << (16 * h);
                            }
                        } else {
                            const int k = c0 + j, d = k - xo;
                            if (used && d >= 0 && d <= 2 * R)
                                word = split_part<PREC>(cf.c[(dzi * W + dyi) * W + d], p);
                        }
                        v[j] = word;
                    }
                    const uint32_t col = C::BAND_COL0 + (dzi * C::NPARTS + p) * C::BANDCOLS + c0;
                    tc::tmem_st_32x32b_x8(tbase + ((uint32_t)(warp * 32) << 16) + col, v);
                }
        tc::tmem_wait_st();
    }

    // group i -> (tile origin, first output plane)
    auto group_origin = [&](int i, int &x0, int &y0, int &z0) {
        const int t = (int)blockIdx.x + (i / a.groups) * (int)gridDim.x;
        const int g = i % a.groups;
        const int xt = t % a.tiles_x, yt = (t / a.tiles_x) % a.tiles_y, zc = t / (a.tiles_x * a.tiles_y);
        x0 = xt * C::TXO;
        y0 = yt * C::TY;
        z0 = (zc * a.groups + g) * C::NZ;
    };
    auto issue_tma = [&](int i) {
        int x0, y0, z0;
        group_origin(i, x0, y0, z0);
        ptx::mbar_arrive_expect_tx(&full[i & 1], C::STG_BYTES);
        ptx::tma_load_3d(stg + (size_t)(i & 1) * (C::STG_BYTES / 4), &tmap, x0, y0, z0, &full[i & 1]);
    };
    if (tid == 0) {
        ptx::prefetch_tmap(&tmap);
        for (int i = 0; i < 2 && i < ng; ++i) issue_tma(i);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    int issued = 0, drained = 0;  // MMA groups issued by thread 0 / drained by the epilogue

    auto epilogue = [&](int j) -> bool {
        const bool ok = ptx::mbar_wait_bounded(&mmad[j & 1], (uint32_t)(j >> 1) & 1u, err);
        if (!ok) *abort_flag = 1;
        __syncthreads();
        if (*abort_flag) return false;
        tc::fence_after_sync();
        ++drained;
        int x0, y0, z0;
        group_origin(j, x0, y0, z0);
        for (int zl = 0; zl < C::NZ; ++zl) {
            uint32_t r[32];
            tc::tmem_ld_32x32b_x32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)((j & 1) * C::N + zl * C::YP), r);
            tc::tmem_wait_ld();
            float *row = dsm + (warp * 32 + lane) * C::DSM_LD;
#pragma unroll
            for (int c = 0; c < 32; ++c) row[c] = __uint_as_float(r[c]);
            __syncthreads();
            const int z = z0 + zl;
            if (z < a.nz) {
                for (int it = tid; it < C::TXO * C::TY; it += C::NT) {
                    const int xl = it % C::TXO, yl = it / C::TXO;
                    const int x = x0 + xl, y = y0 + yl;
                    if (x < a.nx && y < a.ny) {
                        float s = 0.f;
#pragma unroll
                        for (int dyi = 0; dyi < W; ++dyi) s += dsm[(dyi * C::TXO + xl) * C::DSM_LD + yl + dyi];
                        a.out[(int64_t)z * a.opz + (int64_t)y * a.opy + x] = s;
                    }
                }
            }
            __syncthreads();
        }
        tc::fence_before_sync();
        return true;
    };

    bool alive = true;
    for (int i = 0; i < ng && alive; ++i) {
        const int s = i & 1;
        // 1. the FP32 box of group i has landed
        if (!ptx::mbar_wait_bounded(&full[s], (uint32_t)(i >> 1) & 1u, err)) *abort_flag = 1;
        // 2. convert it to the K-major operand parts (hi, lo)
        if (!*abort_flag) {
            const float *src = stg + (size_t)s * (C::STG_BYTES / 4);
            unsigned char *dst = conv + (size_t)s * C::CONV_BYTES;
            constexpr int NCH = C::K / C::KC;  // 16-byte chunks per line
            for (int it = tid; it < C::NL * NCH; it += C::NT) {
                const int kc = it % NCH, n = it / NCH;
                const float *p = src + n * C::K + kc * C::KC;
                float v[8];
                const float4 q0 = *reinterpret_cast<const float4 *>(p);
                v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
                if constexpr (C::KC == 8) {
                    const float4 q1 = *reinterpret_cast<const float4 *>(p + 4);
                    v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
                }
#pragma unroll
                for (int part = 0; part < C::NPARTS; ++part) {
                    uint4 o;
                    if constexpr (C::BF) {
                        uint32_t w4[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h)
                            w4[h] = split_part<PREC>(v[2 * h], part) | (split_part<PREC>(v[2 * h + 1], part) << 16);
                        o = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                    } else {
                        o = make_uint4(split_part<PREC>(v[0], part), split_part<PREC>(v[1], part),
                                       split_part<PREC>(v[2], part), split_part<PREC>(v[3], part));
                    }
                    *reinterpret_cast<uint4 *>(dst + (size_t)part * C::PART_BYTES + ((size_t)kc * C::NL + n) * 16) = o;
                }
            }
            ptx::fence_proxy_async_smem();  // generic writes -> tensor-core reads
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (*abort_flag) { alive = false; break; }
        // 3. thread 0: refill the staging buffer, issue group i's MMAs
        if (tid == 0) {
            if (i + 2 < ng) issue_tma(i + 2);
            const uint32_t dcol = tbase + (uint32_t)(s * C::N);
            const uint32_t cbase = ptx::smem_u32(conv + (size_t)s * C::CONV_BYTES);
            uint32_t acc = 0;
            for (int dzi = 0; dzi < W; ++dzi) {
#pragma unroll
                for (int pr = 0; pr < C::NPROD; ++pr) {
                    const int pa = pr == 2 ? 1 : 0;  // band part
                    const int pb = pr == 1 ? 1 : 0;  // data part
#pragma unroll
                    for (int kk = 0; kk < C::K / C::KSTEP; ++kk) {
                        const uint32_t acol = tbase + C::BAND_COL0 + (dzi * C::NPARTS + pa) * C::BANDCOLS +
                                              kk * (C::KSTEP * C::ELT / 4);
                        const uint32_t baddr = cbase + pb * C::PART_BYTES + (dzi * C::YP) * 16 +
                                               kk * (C::KSTEP / C::KC) * C::NL * 16;
                        const uint64_t bdesc = tc::smem_desc(baddr, C::NL * 16, 128);
                        if constexpr (C::BF)
                            tc::mma_bf16_ts(dcol, acol, bdesc, C::IDESC, acc);
                        else
                            tc::mma_tf32_ts(dcol, acol, bdesc, C::IDESC, acc);
                        acc = 1;
                    }
                }
            }
            tc::mma_commit(&mmad[s]);
            ++issued;
        }
        // 4. drain the previous group's accumulator
        if (i >= 1 && !epilogue(i - 1)) { alive = false; break; }
    }
    if (alive && ng >= 1) epilogue(ng - 1);

    // teardown: no MMA may still write TMEM when it is freed
    if (tid == 0 && issued > drained) {
        for (int j = drained; j < issued; ++j) ptx::mbar_wait_bounded(&mmad[j & 1], (uint32_t)(j >> 1) & 1u, err);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, 512);
    }
}

int g_num_sms = 0;

int num_sms()
{
    if (g_num_sms == 0) {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_num_sms = n > 0 ? n : 152;
    }
    return g_num_sms;
}

template <int R, int PREC>
cudaError_t launch_r(const Sweep &s, const CUtensorMap &map, int groups)
{
    using C = Cfg<R, PREC>;
    if constexpr (!C::OK) {
        return cudaErrorNotSupported;
    } else {
        BoxCoef cf{};
        const int w = 2 * R + 1;
        for (int i = 0; i < w * w * w; ++i) cf.c[i] = s.coeffs[i];
        TcArgs a;
        a.out = s.out;
        a.opy = s.opy;
        a.opz = s.opz;
        a.nx = (int)s.nx;
        a.ny = (int)s.ny;
        a.nz = (int)s.nz;
        a.tiles_x = (int)((s.nx + C::TXO - 1) / C::TXO);
        a.tiles_y = (int)((s.ny + C::TY - 1) / C::TY);
        const int zgroups = (int)((s.nz + C::NZ - 1) / C::NZ);
        a.groups = groups < zgroups ? groups : zgroups;
        const int zchunks = (zgroups + a.groups - 1) / a.groups;
        a.tiles = a.tiles_x * a.tiles_y * zchunks;
        auto kern = box_tc_kernel<R, PREC>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        const int grid = a.tiles < num_sms() ? a.tiles : num_sms();
        kern<<<grid, C::NT, C::SMEM, s.stream>>>(map, cf, a, device_error_word());
        return cudaGetLastError();
    }
}

// Variants: z-groups per tile (the z extent of a tile is groups * NZ planes).
constexpr int kGroups[] = {16, 8, 32, 4};
constexpr int kNumVariants = sizeof(kGroups) / sizeof(int);

template <int PREC>
cudaError_t launch_prec(const Sweep &s, const CUtensorMap &map, int v)
{
    const int g = kGroups[v];
    switch (s.r) {
        case 1: return launch_r<1, PREC>(s, map, g);
        case 2: return launch_r<2, PREC>(s, map, g);
        case 3: return launch_r<3, PREC>(s, map, g);
        case 4: return launch_r<4, PREC>(s, map, g);
        default: return cudaErrorInvalidValue;
    }
}

template <int PREC>
void box_dims(int r, int *bx, int *by, int *bz)
{
#define MMS_DIMS(RR)                                  \
    case RR:                                          \
        *bx = Cfg<RR, PREC>::K;                       \
        *by = Cfg<RR, PREC>::YP;                      \
        *bz = Cfg<RR, PREC>::ZS;                      \
        return;
    switch (r) {
        MMS_DIMS(1)
        MMS_DIMS(2)
        MMS_DIMS(3)
        MMS_DIMS(4)
        default: *bx = *by = *bz = 0;
    }
#undef MMS_DIMS
}

template <int PREC>
bool supported_r(int r)
{
    switch (r) {
        case 1: return Cfg<1, PREC>::OK;
        case 2: return Cfg<2, PREC>::OK;
        case 3: return Cfg<3, PREC>::OK;
        case 4: return Cfg<4, PREC>::OK;
        default: return false;
    }
}

int prec_of(int path)
{
    switch (path) {
        case MMS_PATH_TF32: return P_TF32;
        case MMS_PATH_3XTF32: return P_3XTF32;
        case MMS_PATH_BF16X3: return P_BF16X3;
        default: return -1;
    }
}

}  // namespace

int band_tc_supported(int shape, int r, int path)
{
    if (shape != MMS_BOX) return 0;
    switch (prec_of(path)) {
        case P_TF32: return supported_r<P_TF32>(r);
        case P_3XTF32: return supported_r<P_3XTF32>(r);
        case P_BF16X3: return supported_r<P_BF16X3>(r);
        default: return 0;
    }
}

int band_tc_variants(int shape, int r, int path) { return band_tc_supported(shape, r, path) ? kNumVariants : 0; }

void band_tc_box(int shape, int r, int path, int v, int *bx, int *by, int *bz)
{
    (void)shape;
    (void)v;
    switch (prec_of(path)) {
        case P_TF32: box_dims<P_TF32>(r, bx, by, bz); return;
        case P_3XTF32: box_dims<P_3XTF32>(r, bx, by, bz); return;
        case P_BF16X3: box_dims<P_BF16X3>(r, bx, by, bz); return;
        default: *bx = *by = *bz = 0;
    }
}

cudaError_t launch_band_tc(const Sweep &s, int path, const CUtensorMap &map, int v)
{
    if (v < 0 || v >= kNumVariants) return cudaErrorInvalidValue;
    switch (prec_of(path)) {
        case P_TF32: return launch_prec<P_TF32>(s, map, v);
        case P_3XTF32: return launch_prec<P_3XTF32>(s, map, v);
        case P_BF16X3: return launch_prec<P_BF16X3>(s, map, v);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mms
