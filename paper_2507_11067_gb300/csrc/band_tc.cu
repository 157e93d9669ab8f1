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
// Pipeline (persistent CTAs, one per SM, 16 warps in four roles, double
// buffers handed over by mbarriers): TMA stages the FP32 box of group i+1
// while converter warps turn group i into operand parts, one thread issues
// the MMAs of group i-1 and the epilogue warps drain the TMEM accumulator
// of group i-2.
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
    static constexpr int NT = 512;                   // 16 warps, 4 per TMEM lane quarter
    static constexpr int DSM_LD = 132;               // epilogue: [row y][lane] floats, two planes
    static constexpr int DSM_PLANE = YP * DSM_LD;
    static constexpr int DSM_BYTES = 2 * DSM_PLANE * 4;
    static constexpr int BAND_COL0 = 2 * N;          // TMEM: D0 | D1 | bands
    static constexpr uint32_t IDESC = tc::instr_desc(BF ? 1u : 2u, 128, N);
    // shared memory: [stg0 stg1 | conv0 conv1 | dsm | barriers, tmem slot, flag]
    static constexpr size_t OFF_CONV = 2 * (size_t)STG_BYTES;
    static constexpr size_t OFF_DSM = OFF_CONV + 2 * (size_t)CONV_BYTES;
    static constexpr size_t OFF_BAR = OFF_DSM + DSM_BYTES;
    static constexpr size_t SMEM = 128 + OFF_BAR + 128;
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
    int vec;                      // 16-byte output rows: float4 stores
    int tiles_x, tiles_y, tiles;  // tiles = tiles_x * tiles_y * zchunks
    int groups;                   // groups (of NZ planes) per tile
};

// Warp roles (16 warps): 0 = TMA producer, 1 = MMA issuer (and TMEM owner),
// 2..7 = converters (FP32 box -> operand parts), 8..15 = epilogue (two per
// TMEM lane quarter).  Roles hand buffers to each other through mbarriers,
// so TMA, conversion, MMA and epilogue of different groups overlap.
constexpr int kConvWarps = 6, kConvWarp0 = 2, kEpiWarps = 8, kEpiWarp0 = 8;

__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int R, int PREC>
__global__ void __launch_bounds__(512, 1)
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
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    uint64_t *full_stg = bar, *empty_stg = bar + 2, *full_conv = bar + 4, *empty_conv = bar + 6;
    uint64_t *full_d = bar + 8, *empty_d = bar + 10;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 12);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *epi_fail = abort_flag + 1, *epi_stop = abort_flag + 2;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int my_tiles = a.tiles > (int)blockIdx.x ? (a.tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int ng = my_tiles * a.groups;

    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&full_stg[b], 1);
            ptx::mbar_init(&empty_stg[b], kConvWarps * 32);
            ptx::mbar_init(&full_conv[b], kConvWarps * 32);
            ptx::mbar_init(&empty_conv[b], 1);
            ptx::mbar_init(&full_d[b], 1);
            ptx::mbar_init(&empty_d[b], kEpiWarps);
        }
        ptx::fence_mbar_init();
        *abort_flag = 0;
        *epi_fail = 0;
        *epi_stop = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tmem_slot;

    // Banded coefficient operand, written once by the first warp of each lane
    // quarter: lane (dy, x) of part p for plane offset dz.
    if (warp >= kEpiWarp0 && warp < kEpiWarp0 + 4) {
        const int q = warp & 3;
        const int l = q * 32 + lane;
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
                    tc::tmem_st_32x32b_x8(tbase + ((uint32_t)(q * 32) << 16) + col, v);
                }
        tc::tmem_wait_st();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    // group i -> (tile origin, first output plane)
    auto group_origin = [&](int i, int &x0, int &y0, int &z0) {
        const int t = (int)blockIdx.x + (i / a.groups) * (int)gridDim.x;
        const int g = i % a.groups;
        const int xt = t % a.tiles_x, yt = (t / a.tiles_x) % a.tiles_y, zc = t / (a.tiles_x * a.tiles_y);
        x0 = xt * C::TXO;
        y0 = yt * C::TY;
        z0 = (zc * a.groups + g) * C::NZ;
    };
    // Bounded wait; on expiry raise the CTA-wide abort flag.
    auto wait = [&](uint64_t *b, uint32_t parity) -> bool {
        if (*abort_flag) return false;
        if (ptx::mbar_wait_bounded(b, parity, err)) return true;
        *abort_flag = 1;
        return false;
    };

    if (warp == 0) {
        // ---------------------------------------------------- TMA producer
        if (lane == 0) {
            ptx::prefetch_tmap(&tmap);
            for (int i = 0; i < ng; ++i) {
                const int s = i & 1;
                if (!wait(&empty_stg[s], ((uint32_t)(i >> 1) & 1u) ^ 1u)) break;
                int x0, y0, z0;
                group_origin(i, x0, y0, z0);
                ptx::mbar_arrive_expect_tx(&full_stg[s], C::STG_BYTES);
                ptx::tma_load_3d(stg + (size_t)s * (C::STG_BYTES / 4), &tmap, x0, y0, z0, &full_stg[s]);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            for (int i = 0; i < ng; ++i) {
                const int s = i & 1;
                const uint32_t ph = (uint32_t)(i >> 1) & 1u;
                if (!wait(&full_conv[s], ph)) break;
                if (!wait(&empty_d[s], ph ^ 1u)) break;
                tc::fence_after_sync();
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
                tc::mma_commit(&full_d[s]);      // accumulator ready for the epilogue
                tc::mma_commit(&empty_conv[s]);  // operand stage may be refilled
            }
            // every issued MMA completes before TMEM is freed at teardown
            if (ng > 0) ptx::mbar_wait_bounded(&empty_conv[(ng - 1) & 1], (uint32_t)((ng - 1) >> 1) & 1u, err);
        }
    } else if (warp < kConvWarp0 + kConvWarps) {
        // -------------------------------------------------------- converters
        const int ct = tid - kConvWarp0 * 32;
        constexpr int CT = kConvWarps * 32;
        for (int i = 0; i < ng; ++i) {
            const int s = i & 1;
            const uint32_t ph = (uint32_t)(i >> 1) & 1u;
            // decisions stay warp-uniform: a failed wait in any lane stops the warp
            bool ok = ptx::mbar_wait_bounded(&full_stg[s], ph, err) &&
                      ptx::mbar_wait_bounded(&empty_conv[s], ph ^ 1u, err);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                *abort_flag = 1;
                break;
            }
            const float *src = stg + (size_t)s * (C::STG_BYTES / 4);
            unsigned char *dst = conv + (size_t)s * C::CONV_BYTES;
            constexpr int NCH = C::K / C::KC;  // 16-byte chunks per line
            for (int it = ct; it < C::NL * NCH; it += CT) {
                const int kc = it % NCH, n = it / NCH;
                const float *p = src + n * C::K + kc * C::KC;
                unsigned char *d0 = dst + ((size_t)kc * C::NL + n) * 16;
                if constexpr (C::BF) {
                    const float4 q0 = *reinterpret_cast<const float4 *>(p);
                    const float4 q1 = *reinterpret_cast<const float4 *>(p + 4);
                    const float v[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
                    uint32_t hi[4], lo[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        // one cvt packs the pair (even k in the low half)
                        const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
                        hi[h] = *reinterpret_cast<const uint32_t *>(&b);
                        const float h0 = __uint_as_float(hi[h] << 16), h1 = __uint_as_float(hi[h] & 0xffff0000u);
                        const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * h] - h0, v[2 * h + 1] - h1);
                        lo[h] = *reinterpret_cast<const uint32_t *>(&l);
                    }
                    *reinterpret_cast<uint4 *>(d0) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4 *>(d0 + C::PART_BYTES) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                } else {
                    const float4 q = *reinterpret_cast<const float4 *>(p);
                    const uint32_t h0 = tf32_rna(q.x), h1 = tf32_rna(q.y), h2 = tf32_rna(q.z), h3 = tf32_rna(q.w);
                    *reinterpret_cast<uint4 *>(d0) = make_uint4(h0, h1, h2, h3);
                    if constexpr (C::NPARTS == 2)
                        *reinterpret_cast<uint4 *>(d0 + C::PART_BYTES) =
                            make_uint4(tf32_rna(q.x - __uint_as_float(h0)), tf32_rna(q.y - __uint_as_float(h1)),
                                       tf32_rna(q.z - __uint_as_float(h2)), tf32_rna(q.w - __uint_as_float(h3)));
                }
            }
            ptx::fence_proxy_async_smem();  // generic writes -> tensor-core reads
            ptx::mbar_arrive(&full_conv[s]);
            ptx::mbar_arrive(&empty_stg[s]);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        // TMEM -> registers -> shared memory, the sum over the 2r+1 lanes
        // (dy, x) with rows shifted by dy, float4 stores.  Lane (dy, x) of
        // column c feeds output row y = c - dy, so it is stored at [y][lane]
        // and the reduction reads four x positions per load.
        const int q = warp & 3, half = (warp - kEpiWarp0) >> 2;
        const int my_lane = q * 32 + lane;
        const int my_dyi = my_lane < C::LANES ? my_lane / C::TXO : 0;
        const int et = tid - kEpiWarp0 * 32;
        constexpr int ET = kEpiWarps * 32;
        constexpr int XQ = C::TXO / 4;
        int plane_ctr = 0;
        for (int i = 0; i < ng; ++i) {
            const int s = i & 1;
            // the epilogue warps share named barriers: they stop together
            if (!ptx::mbar_wait_bounded(&full_d[s], (uint32_t)(i >> 1) & 1u, err)) *epi_fail = 1;
            named_sync(1, ET);
            if (et == 0) *epi_stop = (*epi_fail || *abort_flag) ? 1 : 0;
            named_sync(1, ET);
            if (*epi_stop) {
                *abort_flag = 1;
                break;
            }
            tc::fence_after_sync();
            int x0, y0, z0;
            group_origin(i, x0, y0, z0);
            for (int zl = 0; zl < C::NZ; ++zl, ++plane_ctr) {
                float *dbuf = dsm + (plane_ctr & 1) * C::DSM_PLANE;
                uint32_t r[16];
                tc::tmem_ld_32x32b_x16(tbase + ((uint32_t)(q * 32) << 16) +
                                           (uint32_t)(s * C::N + zl * C::YP + half * 16),
                                       r);
                tc::tmem_wait_ld();
                if (my_lane < C::LANES) {
                    float *dst = dbuf + my_lane;
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const int y = half * 16 + c - my_dyi;
                        if (y >= 0 && y < C::TY) dst[y * C::DSM_LD] = __uint_as_float(r[c]);
                    }
                }
                if (zl == C::NZ - 1) {
                    // all TMEM reads of this accumulator are done: hand it back
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&empty_d[s]);
                }
                named_sync(1, ET);
                const int z = z0 + zl;
                if (z < a.nz) {
                    for (int it = et; it < C::TY * XQ; it += ET) {
                        const int xq = it % XQ, yl = it / XQ;
                        const int y = y0 + yl, x = x0 + 4 * xq;
                        if (y >= a.ny || x >= a.nx) continue;
                        const float *src = dbuf + yl * C::DSM_LD + 4 * xq;
                        float4 acc = *reinterpret_cast<const float4 *>(src);
#pragma unroll
                        for (int dyi = 1; dyi < W; ++dyi) {
                            const float4 t = *reinterpret_cast<const float4 *>(src + dyi * C::TXO);
                            acc.x += t.x; acc.y += t.y; acc.z += t.z; acc.w += t.w;
                        }
                        float *o = a.out + (int64_t)z * a.opz + (int64_t)y * a.opy + x;
                        if (a.vec && x + 3 < a.nx) {
                            *reinterpret_cast<float4 *>(o) = acc;
                        } else {
                            const float v4[4] = {acc.x, acc.y, acc.z, acc.w};
                            for (int k = 0; k < 4 && x + k < a.nx; ++k) o[k] = v4[k];
                        }
                    }
                }
            }
        }
    }

    __syncwarp();  // the single-lane roles reconverge their warps first
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
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
        a.vec = (s.opy % 4 == 0 && s.opz % 4 == 0 && reinterpret_cast<uintptr_t>(s.out) % 16 == 0) ? 1 : 0;
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
