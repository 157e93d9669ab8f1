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
// Pipeline (persistent CTAs, one per SM, warps in four roles, buffers handed
// over by mbarriers): TMA stages the FP32 planes of later groups while
// converter warps turn them into operand parts, two issuer warps take turns
// with the MMAs of groups i and i+1 (one TMEM accumulator each) and the
// epilogue warps drain the accumulator of the group before.
#include <cuda_bf16.h>
#include <stdio.h>

#include "common.cuh"
#include "tc.cuh"

namespace mms {

#ifdef MMS_ROLE_TRACE
// Role trace (debug builds only, -DMMS_ROLE_TRACE): cycles each role of the
// first eight CTAs spends waiting on its barriers and in total, summed.
//   [0] producer: wait empty staging, total
//   [1] MMA: wait operands, total, wait accumulator, issuing
//   [2] converter (first lane): wait staging, total, wait operand slot
//   [3] epilogue (first lane): wait accumulator, total, group barriers
__device__ unsigned long long g_role_trace[4][4];
#define MMS_TRACE_ADD(role, slot, v) \
    do { if (blockIdx.x < 8) atomicAdd(&g_role_trace[role][slot], (unsigned long long)(v)); } while (0)
#define MMS_CLOCK() clock64()
extern "C" int mms_role_trace_read(unsigned long long *host, int reset)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;
    if (cudaMemcpyFromSymbol(host, g_role_trace, sizeof(g_role_trace)) != cudaSuccess) return 1;
    if (reset) {
        unsigned long long z[4][4] = {};
        cudaMemcpyToSymbol(g_role_trace, z, sizeof(z));
    }
    return 0;
}
#else
#define MMS_TRACE_ADD(role, slot, v) do { } while (0)
#define MMS_CLOCK() 0ull
#endif

namespace {

enum { P_TF32 = 0, P_3XTF32 = 1, P_BF16X3 = 2 };

constexpr int roundup(int a, int b) { return (a + b - 1) / b * b; }

template <int R, int PREC, bool LDG = false, bool PLANAR = false>
struct Cfg {
    // LDG: converter warps read the FP32 input from global memory themselves
    // (no TMA staging ring); otherwise a producer warp stages it with TMA.
    // PLANAR: the stencil has no z extent (2D in each plane of the padded
    // grid, coefficients [dy][dx]): the x/y pass of the star on tensor cores.
    static constexpr int RZ = PLANAR ? 0 : R;
    static constexpr int WZ = 2 * RZ + 1;
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
    static constexpr int BAND_TOTAL = WZ * NPARTS * BANDCOLS;
    // staged rows per plane: 32, or 36 at radius 2, whose 32 output rows
    // per tile divide the usual power-of-two extents (N = 4 x 36 = 144 is
    // a legal MMA N); elsewhere (other radii, and 3xTF32, whose larger bands
    // leave room for 2 planes per group) N would not be a multiple of 16
    static constexpr int YP = (R == 2 && PREC != P_3XTF32) ? 36 : 32;
    static constexpr int TY = YP - 2 * R;            // output rows per tile
    static constexpr int NZ = (2 * 4 * YP + BAND_TOTAL <= 512)   ? 4
                              : (2 * 3 * YP + BAND_TOTAL <= 512) ? 3
                              : (2 * 2 * YP + BAND_TOTAL <= 512) ? 2
                                                                 : 1;
    static constexpr bool FITS_TMEM = 2 * NZ * YP + BAND_TOTAL <= 512 && LANES <= 128;
    static constexpr int N = NZ * YP;                // MMA N (lines per group)
    // Planes are staged and converted once, in chunks of NZ planes.  Group g
    // of a tile reads planes [g NZ, g NZ + NZ + 2R) = chunks g .. g + H; the
    // converted chunks live in a ring of CR slots plus H duplicate slots (a
    // chunk in slot s < H is also written to slot CR + s), so every window of
    // H + 1 consecutive chunks is contiguous and one descriptor spans it.
    static constexpr int H = (2 * RZ + NZ - 1) / NZ;
    static constexpr int CR = H + 2;
    static constexpr int CHUNK_LINES = NZ * YP;
    static constexpr int RING_LINES = (CR + H) * CHUNK_LINES;
    static constexpr int PART_BYTES = RING_LINES * K * ELT;  // one operand part, whole ring
    static constexpr int CONV_BYTES = PART_BYTES * NPARTS;
    static constexpr int STG_BYTES = CHUNK_LINES * K * 4;     // FP32 TMA staging of one chunk
    // epilogue: one [row y + 2R][lane] float tile per epilogue warp group.
    // A row stride of 0 mod 32 words puts lane l in bank l whatever its row,
    // so the scattered stores are conflict-free; 2R spare rows take the
    // values that fall outside the tile, so every store is unconditional; the
    // reduction pads its x quads to a multiple of 8 so that 8 consecutive
    // items read 8 different bank groups.
    static constexpr int DSM_LD = 128;
    static constexpr int XQ = TXO / 4, XQP = (XQ + 7) / 8 * 8;
    static constexpr int DSM_ROWS = YP + 2 * R;
    static constexpr int DSM_GROUP = DSM_ROWS * DSM_LD;  // floats per epilogue group
    static constexpr int BAND_COL0 = 2 * N;          // TMEM: D0 | D1 | bands
    static constexpr uint32_t IDESC = tc::instr_desc(BF ? 1u : 2u, 128, N);
    // shared memory: [conv ring | dsm | staging ring | barriers, tmem slot, flags]
    static constexpr size_t BUDGET = 227 * 1024;
    static constexpr size_t BASE = (size_t)CONV_BYTES + 1024 + 512;
    static constexpr size_t GRP = (size_t)DSM_GROUP * 4;
    // epilogue warp groups (4 warps, one per TMEM lane quarter, each owns whole
    // planes of the accumulator): as many as the planes and shared memory allow
    static constexpr size_t STG_MIN = LDG ? 0 : 2 * (size_t)STG_BYTES;
    static constexpr int EGF = BASE + 4 * GRP + STG_MIN <= BUDGET   ? 4
                               : BASE + 3 * GRP + STG_MIN <= BUDGET ? 3
                               : BASE + 2 * GRP + STG_MIN <= BUDGET ? 2
                                                                   : 1;
    static constexpr int EG = EGF < NZ ? EGF : NZ;
    static constexpr int DSM_BYTES = EG * DSM_GROUP * 4;
    static constexpr int NCONV = LDG ? 5 : 4;        // converter warps: (0,) 2, 3 and the last two
    static constexpr int NWARPS = 4 + 4 * EG + 3;   // + the second MMA issuer (last warp)
    static constexpr int NT = 32 * NWARPS;
    static constexpr size_t FIXED = BASE + DSM_BYTES;
    static constexpr int NST = LDG                                           ? 0
                               : FIXED + 4 * (size_t)STG_BYTES <= BUDGET   ? 4
                               : FIXED + 3 * (size_t)STG_BYTES <= BUDGET ? 3
                                                                         : 2;
    static constexpr size_t OFF_DSM = CONV_BYTES;
    static constexpr size_t OFF_STG = OFF_DSM + DSM_BYTES;
    static constexpr size_t OFF_BAR = OFF_STG + (size_t)NST * STG_BYTES;
    static constexpr size_t SMEM = 1024 + OFF_BAR + 512;
    static constexpr bool OK = FITS_TMEM && SMEM <= BUDGET && RING_LINES * 16 < (1 << 18);
    // FP32 staging rows of exactly 128 bytes are loaded with the TMA 128-byte
    // swizzle: 16-byte chunk q of line n sits at chunk q ^ (n & 7), so the
    // converters' column reads across 8 lines hit 8 different bank groups.
    static constexpr bool SWZ = K * 4 == 128;
    static_assert(SWZ == (K * 4 == 128) && N % 16 == 0 && N <= 256, "MMA N");
    static_assert(YP == 32 || YP == 36, "the epilogue loads 32 or 36 accumulator columns");
    static_assert(STG_BYTES % 1024 == 0 && CONV_BYTES % 1024 == 0 && PART_BYTES % 16 == 0, "align");
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
    const float *in;              // padded input (read directly by LDG converters)
    int64_t ipy, ipz;
    int X, Y, Z;                  // padded extents
    float *out;
    int64_t opy, opz;
    int nx, ny, nz;
    int vec;                      // 16-byte output rows: float4 stores
    int tiles_x, tiles_y, tiles;  // tiles = tiles_x * tiles_y * zchunks
    int groups;                   // groups (of NZ planes) per tile
    int zoff;                     // input plane of output plane 0 (R for a z-padded grid, 0 for planar shapes)
};

// Warp roles: 0 = TMA producer, 1 = MMA issuer of the even groups (and TMEM
// owner), the last warp = MMA issuer of the odd groups, 2, 3 and the two
// warps before the last = converters (FP32 box -> operand parts),
// 4 .. 4+4EG-1 = epilogue, EG groups of four warps (warp w reaches TMEM lane
// quarter w % 4); group e drains planes e, e+EG, ... of each accumulator.
// Roles hand buffers to each other through mbarriers, so TMA, conversion,
// MMA and epilogue of different groups overlap.

__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// 16 bytes of the padded input at (xi, yi, zi), zero outside the grid.
__device__ __forceinline__ float4 load_in4(const TcArgs &a, int xi, int yi, int zi)
{
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (yi >= a.Y || zi >= a.Z || xi >= a.X) return v;
    const float *p = a.in + (int64_t)zi * a.ipz + (int64_t)yi * a.ipy + xi;
    if (xi + 3 < a.X) return __ldg(reinterpret_cast<const float4 *>(p));
    v.x = __ldg(p);
    if (xi + 1 < a.X) v.y = __ldg(p + 1);
    if (xi + 2 < a.X) v.z = __ldg(p + 2);
    return v;
}

template <int R, int PREC, bool LDG, bool PLANAR>
__global__ void __launch_bounds__(Cfg<R, PREC, LDG, PLANAR>::NT, 1)
    box_tc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ BoxCoef cf,
                  const __grid_constant__ TcArgs a, unsigned *err)
{
    using C = Cfg<R, PREC, LDG, PLANAR>;
    constexpr int W = C::W;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 1024-byte alignment: the TMA swizzle pattern repeats every 1024 bytes
    unsigned char *smem = smem_raw + ((1024u - (ptx::smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *conv = smem;
    float *dsm = reinterpret_cast<float *>(smem + C::OFF_DSM);
    float *stg = reinterpret_cast<float *>(smem + C::OFF_STG);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    uint64_t *full_stg = bar, *empty_stg = bar + C::NST;
    uint64_t *full_conv = bar + 2 * C::NST, *empty_conv = full_conv + C::CR;
    uint64_t *full_d = empty_conv + C::CR, *empty_d = full_d + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(empty_d + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *epi_fail = abort_flag + 1;  // [EG][2], by epilogue group and accumulator parity
    constexpr int CT = C::NCONV * 32;           // converter threads
    constexpr int NEPI = 4 * C::EG;             // epilogue warps

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int my_tiles = a.tiles > (int)blockIdx.x ? (a.tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int G = a.groups, CPT = a.groups + C::H;  // groups and chunks per tile
    const int ng = my_tiles * G, nch = my_tiles * CPT;

    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < C::NST; ++b) {
            ptx::mbar_init(&full_stg[b], 1);
            ptx::mbar_init(&empty_stg[b], CT);
        }
        for (int b = 0; b < C::CR; ++b) {
            ptx::mbar_init(&full_conv[b], CT);
            ptx::mbar_init(&empty_conv[b], C::H + 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&full_d[b], 1);
            ptx::mbar_init(&empty_d[b], NEPI);
        }
        ptx::fence_mbar_init();
        *abort_flag = 0;
        for (int e = 0; e < 2 * C::EG; ++e) epi_fail[e] = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tmem_slot;

    // Banded coefficient operand, written once by the first warp of each lane
    // quarter: lane (dy, x) of part p for plane offset dz.
    if (warp >= 4 && warp < 8) {
        const int q = warp & 3;
        const int l = q * 32 + lane;
        const bool used = l < C::LANES;
        const int dyi = used ? l / C::TXO : 0, xo = used ? l % C::TXO : 0;
        for (int dzi = 0; dzi < C::WZ; ++dzi)
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

    // tile (per CTA, tl-th) -> column origin and first plane of its z chunk
    auto tile_origin = [&](int tl, int &x0, int &y0, int &zt) {
        const int t = (int)blockIdx.x + tl * (int)gridDim.x;
        const int xt = t % a.tiles_x, yt = (t / a.tiles_x) % a.tiles_y, zc = t / (a.tiles_x * a.tiles_y);
        x0 = xt * C::TXO;
        y0 = yt * C::TY;
        zt = zc * G * C::NZ;
    };
    // Bounded wait of the producer and MMA roles; on expiry raise the abort flag.
    [[maybe_unused]] unsigned long long waited = 0;  // role trace only
    auto wait = [&](uint64_t *b, uint32_t parity) -> bool {
        if (*abort_flag) return false;
        const unsigned long long t0 = MMS_CLOCK();
        const bool done = ptx::mbar_wait_bounded(b, parity, err);
        waited += MMS_CLOCK() - t0;
        if (done) return true;
        *abort_flag = 1;
        return false;
    };

    if (warp == 0 && !LDG) {
        // ------------------------------------------- TMA producer: chunk k
        // (whole warp waits, one elected lane issues)
        const bool leader = ptx::elect_one();
        [[maybe_unused]] const unsigned long long tstart = MMS_CLOCK();
        if (leader) ptx::prefetch_tmap(&tmap);
        for (int k = 0; k < nch; ++k) {
            constexpr int NSTD = C::NST > 0 ? C::NST : 1;  // (this branch only runs with a ring)
            const int st = k % NSTD;
            const bool ok = wait(&empty_stg[st], ((uint32_t)(k / NSTD) & 1u) ^ 1u);
            if (!__all_sync(0xffffffffu, ok)) {
                *abort_flag = 1;
                break;
            }
            if (leader) {
                int x0, y0, zt;
                tile_origin(k / CPT, x0, y0, zt);
                ptx::mbar_arrive_expect_tx(&full_stg[st], C::STG_BYTES);
                ptx::tma_load_3d(stg + (size_t)st * (C::STG_BYTES / 4), &tmap, x0, y0,
                                 zt + (k % CPT) * C::NZ + a.zoff, &full_stg[st]);
            }
            __syncwarp();
        }
        if (lane == 0) {
            MMS_TRACE_ADD(0, 0, waited);
            MMS_TRACE_ADD(0, 1, MMS_CLOCK() - tstart);
        }
    } else if (warp == 1 || warp == C::NWARPS - 1) {
        // ----------------------------------------------------- MMA issuers
        // Two warps alternate groups: warp 1 issues the even groups into
        // accumulator 0, the last warp the odd ones into accumulator 1.  A
        // warp's barrier polls wait behind its own MMAs still queued, so a
        // single issuer leaves the tensor pipe idle at every group boundary;
        // with two, one warp's queued MMAs cover the other's polls.  The
        // whole warp runs the loop and waits; one elected lane issues.
        const int s = warp == 1 ? 0 : 1;
        const bool leader = ptx::elect_one();
        [[maybe_unused]] const unsigned long long tstart = MMS_CLOCK();
        [[maybe_unused]] unsigned long long wconv = 0, wacc = 0, tissue = 0;
        int last = -1;  // last group this warp issued
        for (int i = s; i < ng; i += 2) {
            const int g = i % G;
            const int kg = (i / G) * CPT + g;  // first chunk of this group's window
            bool ok = true;
            unsigned long long w0 = waited;
            for (int h = 0; h <= C::H && ok; ++h)
                ok = wait(&full_conv[(kg + h) % C::CR], (uint32_t)((kg + h) / C::CR) & 1u);
            wconv += waited - w0;
            w0 = waited;
            ok = ok && wait(&empty_d[s], ((uint32_t)(i >> 1) & 1u) ^ 1u);
            wacc += waited - w0;
            // every lane takes the same decision
            if (!__all_sync(0xffffffffu, ok)) {
                *abort_flag = 1;
                break;
            }
            [[maybe_unused]] const unsigned long long ti = MMS_CLOCK();
            tc::fence_after_sync();
            if (leader) {
                const uint32_t dcol = tbase + (uint32_t)(s * C::N);
                const uint32_t cbase = ptx::smem_u32(conv) + (uint32_t)((kg % C::CR) * C::CHUNK_LINES * 16);
                // one descriptor per group; each MMA adds a constant (>> 4) to its start field
                const uint64_t d0 = tc::smem_desc(cbase, C::RING_LINES * 16, 128);
                const uint32_t a0 = tbase + C::BAND_COL0;
#pragma unroll
                for (int dzi = 0; dzi < C::WZ; ++dzi) {
#pragma unroll
                    for (int pr = 0; pr < C::NPROD; ++pr) {
                        const int pa = pr == 2 ? 1 : 0;  // band part
                        const int pb = pr == 1 ? 1 : 0;  // data part
#pragma unroll
                        for (int kk = 0; kk < C::K / C::KSTEP; ++kk) {
                            const uint32_t acol = a0 + (dzi * C::NPARTS + pa) * C::BANDCOLS + kk * (C::KSTEP * C::ELT / 4);
                            const uint64_t bdesc = d0 + (uint64_t)((pb * C::PART_BYTES + (dzi * C::YP) * 16 +
                                                                    kk * (C::KSTEP / C::KC) * C::RING_LINES * 16) >> 4);
                            const uint32_t acc = (dzi | pr | kk) ? 1u : 0u;
                            if constexpr (C::BF)
                                tc::mma_bf16_ts(dcol, acol, bdesc, C::IDESC, acc);
                            else
                                tc::mma_tf32_ts(dcol, acol, bdesc, C::IDESC, acc);
                        }
                    }
                }
                tc::mma_commit(&full_d[s]);  // accumulator ready for the epilogue
                // A chunk slot is free again after H+1 arrivals: one from every
                // group of the tile that reads the chunk, once its MMAs are
                // done, and, for the chunks at the tile's ends that fewer
                // groups read, the missing ones from their first reader.
                for (int h = 0; h <= C::H; ++h) {
                    const int c = g + h;  // tile-local chunk
                    const int first = c - C::H > 0 ? c - C::H : 0;
                    const int nread = (c < G - 1 ? c : G - 1) - first + 1;
                    const int n = g == first ? C::H + 2 - nread : 1;
                    for (int j = 0; j < n; ++j) tc::mma_commit(&empty_conv[(kg + h) % C::CR]);
                }
            }
            __syncwarp();
            last = i;
            tissue += MMS_CLOCK() - ti;
        }
        // every MMA this warp issued completes before TMEM is freed at teardown
        if (last >= 0) ptx::mbar_wait_bounded(&full_d[s], (uint32_t)(last >> 1) & 1u, err);
        if (lane == 0) {
            MMS_TRACE_ADD(1, 0, wconv);
            MMS_TRACE_ADD(1, 1, MMS_CLOCK() - tstart);
            MMS_TRACE_ADD(1, 2, wacc);
            MMS_TRACE_ADD(1, 3, tissue);
        }
    } else if (warp < 4 || warp >= 4 + NEPI) {
        // -------------------------------------------- converters: chunk k
        const int cw = warp == 0 ? C::NCONV - 1 : warp < 4 ? warp - 2 : warp - 2 - NEPI;
        const int ct = cw * 32 + lane;
        constexpr int NCH = C::K / C::KC;  // 16-byte operand chunks per line
        [[maybe_unused]] const unsigned long long tstart = MMS_CLOCK();
        [[maybe_unused]] unsigned long long wstg = 0, wslot = 0;
        constexpr int NV4 = C::KC / 4;  // FP32 float4 per operand chunk (2 for BF16, 1 for TF32)
        constexpr int IPT = (C::CHUNK_LINES * NCH + CT - 1) / CT;  // items per thread
        for (int k = 0; k < nch; ++k) {
            const int sl = k % C::CR;
            const int st = LDG ? 0 : k % (C::NST > 0 ? C::NST : 1);
            // operand values of this thread's items, from global memory (LDG)
            // or from the TMA staging ring
            float4 in4[IPT][NV4];
            if constexpr (LDG) {
                int x0, y0, zt;
                tile_origin(k / CPT, x0, y0, zt);
                const int zc = zt + (k % CPT) * C::NZ + a.zoff;
#pragma unroll
                for (int t = 0; t < IPT; ++t) {
                    const int it = ct + t * CT;
                    const int n = it % C::CHUNK_LINES, kc = it / C::CHUNK_LINES;
#pragma unroll
                    for (int q = 0; q < NV4; ++q)
                        in4[t][q] = it < C::CHUNK_LINES * NCH
                                        ? load_in4(a, x0 + kc * C::KC + 4 * q, y0 + n % C::YP, zc + n / C::YP)
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            // decisions stay warp-uniform: a failed wait in any lane stops the warp
            [[maybe_unused]] const unsigned long long t0 = MMS_CLOCK();
            constexpr int NSTD = C::NST > 0 ? C::NST : 1;
            bool ok = LDG ? true : ptx::mbar_wait_bounded(&full_stg[st], (uint32_t)(k / NSTD) & 1u, err);
            [[maybe_unused]] const unsigned long long t1 = MMS_CLOCK();
            ok = ok && ptx::mbar_wait_bounded(&empty_conv[sl], ((uint32_t)(k / C::CR) & 1u) ^ 1u, err);
            wstg += t1 - t0;
            wslot += MMS_CLOCK() - t1;
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                *abort_flag = 1;
                break;
            }
            const float *src = stg + (size_t)st * (C::STG_BYTES / 4);
            const int line0 = sl * C::CHUNK_LINES;
            const bool dup = sl < C::H;
            // lines fastest: a warp converts one 16-byte chunk column of 32
            // consecutive lines, so its stores are contiguous
#pragma unroll
            for (int t = 0; t < IPT; ++t) {
                const int it = ct + t * CT;
                if (it >= C::CHUNK_LINES * NCH) break;
                const int n = it % C::CHUNK_LINES, kc = it / C::CHUNK_LINES;
                unsigned char *d0 = conv + ((size_t)kc * C::RING_LINES + line0 + n) * 16;
                if constexpr (!LDG) {
                    const float *line = src + n * C::K;
#pragma unroll
                    for (int q = 0; q < NV4; ++q) {
                        // swizzled staging: 16-byte chunk j of line n sits at j ^ (n & 7)
                        const int j = kc * NV4 + q;
                        const int pj = C::SWZ ? (j ^ (n & 7)) : j;
                        in4[t][q] = *reinterpret_cast<const float4 *>(line + 4 * pj);
                    }
                }
                uint4 o[2];
                if constexpr (C::BF) {
                    const float4 q0 = in4[t][0], q1 = in4[t][NV4 - 1];
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
                    o[0] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    o[1] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                } else {
                    const float4 q = in4[t][0];
                    const uint32_t h0 = tf32_rna(q.x), h1 = tf32_rna(q.y), h2 = tf32_rna(q.z), h3 = tf32_rna(q.w);
                    o[0] = make_uint4(h0, h1, h2, h3);
                    if constexpr (C::NPARTS == 2)
                        o[1] = make_uint4(tf32_rna(q.x - __uint_as_float(h0)), tf32_rna(q.y - __uint_as_float(h1)),
                                          tf32_rna(q.z - __uint_as_float(h2)), tf32_rna(q.w - __uint_as_float(h3)));
                }
#pragma unroll
                for (int part = 0; part < C::NPARTS; ++part) {
                    *reinterpret_cast<uint4 *>(d0 + (size_t)part * C::PART_BYTES) = o[part];
                    if (dup)
                        *reinterpret_cast<uint4 *>(d0 + (size_t)part * C::PART_BYTES +
                                                   (size_t)C::CR * C::CHUNK_LINES * 16) = o[part];
                }
            }
            ptx::fence_proxy_async_smem();  // generic writes -> tensor-core reads
            ptx::mbar_arrive(&full_conv[sl]);
            if (!LDG) ptx::mbar_arrive(&empty_stg[st]);
        }
        if (ct == 0) {
            MMS_TRACE_ADD(2, 0, wstg);
            MMS_TRACE_ADD(2, 1, MMS_CLOCK() - tstart);
            MMS_TRACE_ADD(2, 2, wslot);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        // TMEM -> registers -> shared memory, the sum over the 2r+1 lanes
        // (dy, x) with rows shifted by dy, float4 stores.  Lane (dy, x) of
        // column c feeds output row y = c - dy, so it is stored at
        // [y + 2R][lane] and the reduction reads four x positions per load.
        const int eg = (warp - 4) >> 2, q = warp & 3;
        const int my_lane = q * 32 + lane;
        const int my_dyi = my_lane < C::LANES ? my_lane / C::TXO : 0;
        const int et = (warp & 3) * 32 + lane;  // thread index within the group
        float *gbuf = dsm + eg * C::DSM_GROUP;
        float *st_base = gbuf + (2 * R - my_dyi) * C::DSM_LD + my_lane;
        volatile int *fail = epi_fail + 2 * eg;
        bool stop = false;
        [[maybe_unused]] const unsigned long long tstart = MMS_CLOCK();
        [[maybe_unused]] unsigned long long wacc = 0, wbar = 0;
        for (int i = 0; i < ng && !stop; ++i) {
            const int s = i & 1;
            const unsigned long long t0 = MMS_CLOCK();
            if (!ptx::mbar_wait_bounded(&full_d[s], (uint32_t)(i >> 1) & 1u, err)) fail[s] = 1;
            wacc += MMS_CLOCK() - t0;
            tc::fence_after_sync();
            int x0, y0, zt;
            tile_origin(i / G, x0, y0, zt);
            const int z0 = zt + (i % G) * C::NZ;
            for (int zl = eg; zl < C::NZ; zl += C::EG) {
                uint32_t r[C::YP];
                {
                    const uint32_t ta = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(s * C::N + zl * C::YP);
                    uint32_t (&r32)[32] = *reinterpret_cast<uint32_t (*)[32]>(&r[0]);
                    tc::tmem_ld_32x32b_x32(ta, r32);
                    if constexpr (C::YP == 36) {
                        uint32_t (&r4)[4] = *reinterpret_cast<uint32_t (*)[4]>(&r[32]);
                        tc::tmem_ld_32x32b_x4(ta + 32, r4);
                    }
                }
                tc::tmem_wait_ld();
                if (zl + C::EG >= C::NZ) {
                    // this warp's last read of the accumulator: hand it back
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&empty_d[s]);
                }
#pragma unroll
                for (int c = 0; c < C::YP; ++c) st_base[c * C::DSM_LD] = __uint_as_float(r[c]);
                [[maybe_unused]] const unsigned long long tb = MMS_CLOCK();
                named_sync(1 + eg, 128);
                wbar += MMS_CLOCK() - tb;
                // a timed-out wait (any thread of the group) was recorded before
                // the group's first barrier, in the flag of this accumulator
                // parity, which no thread writes again before all have read it:
                // the four warps take the same decision and stop together
                if (zl == eg && fail[s]) {
                    stop = true;
                    *abort_flag = 1;
                    break;
                }
                const int z = z0 + zl;
                if (z < a.nz) {
                    for (int it = et; it < C::TY * C::XQP; it += 128) {
                        const int xq = it % C::XQP, yl = it / C::XQP;
                        const int y = y0 + yl, x = x0 + 4 * xq;
                        if (xq >= C::XQ || y >= a.ny || x >= a.nx) continue;
                        const float *src = gbuf + (2 * R + yl) * C::DSM_LD + 4 * xq;
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
                named_sync(1 + eg, 128);  // the tile is free for the next plane
            }
        }
        if (warp == 4 && lane == 0) {
            MMS_TRACE_ADD(3, 0, wacc);
            MMS_TRACE_ADD(3, 1, MMS_CLOCK() - tstart);
            MMS_TRACE_ADD(3, 2, wbar);
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

template <int R, int PREC, bool LDG, bool PLANAR = false>
cudaError_t launch_r(const Sweep &s, const CUtensorMap &map, int groups)
{
    using C = Cfg<R, PREC, LDG, PLANAR>;
    if constexpr (!C::OK) {
        return cudaErrorNotSupported;
    } else {
        BoxCoef cf{};
        for (int i = 0; i < C::WZ * C::W * C::W; ++i) cf.c[i] = s.coeffs[i];
        TcArgs a;
        a.in = s.in;
        a.ipy = s.ipy;
        a.ipz = s.ipz;
        a.X = (int)s.nx + 2 * R;
        a.Y = (int)s.ny + 2 * R;
        // planar shapes (a batch of 2D grids) have no z halo; otherwise an
        // output's centre plane is R - RZ planes into the padded grid
        a.Z = (int)s.nz + (is_planar(s.shape) ? 0 : 2 * R);
        a.zoff = is_planar(s.shape) ? 0 : R - C::RZ;
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
        auto kern = box_tc_kernel<R, PREC, LDG, PLANAR>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        const int grid = a.tiles < num_sms() ? a.tiles : num_sms();
        kern<<<grid, C::NT, C::SMEM, s.stream>>>(map, cf, a, device_error_word());
        return cudaGetLastError();
    }
}

// Variants: z-groups per tile (the z extent of a tile is groups * NZ planes)
// times the feed of the converters (TMA staging ring, or direct loads).
constexpr int kGroups[] = {16, 8, 32, 4};
constexpr int kNumGroups = sizeof(kGroups) / sizeof(int);
constexpr int kNumVariants = 2 * kNumGroups;

template <int PREC, bool LDG, bool PLANAR>
cudaError_t launch_feed(const Sweep &s, const CUtensorMap &map, int g)
{
    switch (s.r) {
        case 1: return launch_r<1, PREC, LDG, PLANAR>(s, map, g);
        case 2: return launch_r<2, PREC, LDG, PLANAR>(s, map, g);
        case 3: return launch_r<3, PREC, LDG, PLANAR>(s, map, g);
        case 4: return launch_r<4, PREC, LDG, PLANAR>(s, map, g);
        default: return cudaErrorInvalidValue;
    }
}

template <int PREC, bool PLANAR>
cudaError_t launch_prec(const Sweep &s, const CUtensorMap &map, int v)
{
    const int g = kGroups[v % kNumGroups];
    return v < kNumGroups ? launch_feed<PREC, false, PLANAR>(s, map, g)
                          : launch_feed<PREC, true, PLANAR>(s, map, g);
}

template <int PREC, bool PLANAR>
void box_dims(int r, int *bx, int *by, int *bz, int *swz)
{
#define MMS_DIMS(RR)                                          \
    case RR:                                                  \
        *bx = Cfg<RR, PREC, false, PLANAR>::K;                \
        *by = Cfg<RR, PREC, false, PLANAR>::YP;               \
        *bz = Cfg<RR, PREC, false, PLANAR>::NZ;               \
        *swz = Cfg<RR, PREC, false, PLANAR>::SWZ ? 1 : 0;     \
        return;
    switch (r) {
        MMS_DIMS(1)
        MMS_DIMS(2)
        MMS_DIMS(3)
        MMS_DIMS(4)
        default: *bx = *by = *bz = *swz = 0;
    }
#undef MMS_DIMS
}

template <int PREC, bool PLANAR>
bool supported_r(int r)
{
    switch (r) {
        case 1: return Cfg<1, PREC, false, PLANAR>::OK && Cfg<1, PREC, true, PLANAR>::OK;
        case 2: return Cfg<2, PREC, false, PLANAR>::OK && Cfg<2, PREC, true, PLANAR>::OK;
        case 3: return Cfg<3, PREC, false, PLANAR>::OK && Cfg<3, PREC, true, PLANAR>::OK;
        case 4: return Cfg<4, PREC, false, PLANAR>::OK && Cfg<4, PREC, true, PLANAR>::OK;
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

template <bool PLANAR>
int supported(int r, int path)
{
    switch (prec_of(path)) {
        case P_TF32: return supported_r<P_TF32, PLANAR>(r);
        case P_3XTF32: return supported_r<P_3XTF32, PLANAR>(r);
        case P_BF16X3: return supported_r<P_BF16X3, PLANAR>(r);
        default: return 0;
    }
}

template <bool PLANAR>
cudaError_t launch_tc(const Sweep &s, int path, const CUtensorMap &map, int v)
{
    switch (prec_of(path)) {
        case P_TF32: return launch_prec<P_TF32, PLANAR>(s, map, v);
        case P_3XTF32: return launch_prec<P_3XTF32, PLANAR>(s, map, v);
        case P_BF16X3: return launch_prec<P_BF16X3, PLANAR>(s, map, v);
        default: return cudaErrorInvalidValue;
    }
}

// z part of the star after the tensor-core x/y pass:
//   out(x,y,z) = T(x,y,z) + sum_{dz != 0} cz[dz] in(x+r, y+r, z+r+dz)
// Each thread owns four x positions of one row and marches a z range with a
// register queue of the 2r+1 centre values.
struct ZCoef { float c[2 * kMaxR + 1]; };

template <int R>
__global__ void __launch_bounds__(256)
    star_zpass_kernel(const float *__restrict__ in, int64_t ipy, int64_t ipz, const float *__restrict__ T,
                      int64_t tpy, int64_t tpz, float *__restrict__ out, int64_t opy, int64_t opz, int nx,
                      int ny, int nz, const __grid_constant__ ZCoef cz, int tz, int vec)
{
    constexpr int W = 2 * R + 1;
    const int x = (blockIdx.x * 16 + (threadIdx.x & 15)) * 4;
    const int y = blockIdx.y * 16 + (threadIdx.x >> 4);
    const int zb = blockIdx.z * tz, ze = min(zb + tz, nz);
    if (x >= nx || y >= ny) return;
    const float *col = in + (int64_t)(y + R) * ipy + (x + R);
    const bool full4 = x + 3 < nx;
    auto load4 = [&](const float *p, float (&v)[4]) {
        if (vec && full4 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
            const float4 t = *reinterpret_cast<const float4 *>(p);
            v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = x + k < nx ? p[k] : 0.f;
        }
    };
    float q[W][4];
#pragma unroll
    for (int d = 0; d < W - 1; ++d) load4(col + (int64_t)(zb + d) * ipz, q[d + 1]);  // planes zb-R .. zb+R-1
    for (int z = zb; z < ze; ++z) {
#pragma unroll
        for (int d = 0; d < W - 1; ++d)
#pragma unroll
            for (int k = 0; k < 4; ++k) q[d][k] = q[d + 1][k];
        load4(col + (int64_t)(z + 2 * R) * ipz, q[W - 1]);  // padded plane z + 2R = centre z + R, offset +R
        float t[4], o[4];
        load4(T + (int64_t)z * tpz + (int64_t)y * tpy + x, t);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float acc = t[k];
#pragma unroll
            for (int d = 0; d < W; ++d)
                if (d != R) acc = fmaf(cz.c[d], q[d][k], acc);
            o[k] = acc;
        }
        float *op = out + (int64_t)z * opz + (int64_t)y * opy + x;
        if (vec && full4 && (reinterpret_cast<uintptr_t>(op) & 15) == 0) {
            *reinterpret_cast<float4 *>(op) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (x + k < nx) op[k] = o[k];
        }
    }
}

template <int R>
cudaError_t launch_zpass(const Sweep &s, const float *T, int64_t tpy, int64_t tpz)
{
    ZCoef cz{};
    for (int d = 0; d < 2 * R + 1; ++d) cz.c[d] = s.coeffs[2 * (2 * R + 1) + d];
    const int tz = 64;
    const dim3 grid((unsigned)((s.nx + 63) / 64), (unsigned)((s.ny + 15) / 16), (unsigned)((s.nz + tz - 1) / tz));
    const int vec = (s.ipy % 4 == 0 && s.ipz % 4 == 0 && tpy % 4 == 0 && tpz % 4 == 0 && s.opy % 4 == 0 &&
                     s.opz % 4 == 0)
                        ? 1
                        : 0;
    star_zpass_kernel<R><<<grid, 256, 0, s.stream>>>(s.in, s.ipy, s.ipz, T, tpy, tpz, s.out, s.opy, s.opz,
                                                     (int)s.nx, (int)s.ny, (int)s.nz, cz, tz, vec);
    return cudaGetLastError();
}

}  // namespace

int band_tc_supported(int shape, int r, int path)
{
    // the box runs the 3D kernel; the star's x/y pass and the planar shapes the planar one
    return shape == MMS_BOX ? supported<false>(r, path) : supported<true>(r, path);
}

int band_tc_variants(int shape, int r, int path) { return band_tc_supported(shape, r, path) ? kNumVariants : 0; }

void band_tc_box(int shape, int r, int path, int v, int *bx, int *by, int *bz, int *swz)
{
    (void)v;
    const bool planar = shape != MMS_BOX;
    switch (prec_of(path)) {
        case P_TF32: planar ? box_dims<P_TF32, true>(r, bx, by, bz, swz) : box_dims<P_TF32, false>(r, bx, by, bz, swz); return;
        case P_3XTF32: planar ? box_dims<P_3XTF32, true>(r, bx, by, bz, swz) : box_dims<P_3XTF32, false>(r, bx, by, bz, swz); return;
        case P_BF16X3: planar ? box_dims<P_BF16X3, true>(r, bx, by, bz, swz) : box_dims<P_BF16X3, false>(r, bx, by, bz, swz); return;
        default: *bx = *by = *bz = *swz = 0;
    }
}

size_t band_tc_scratch_bytes(const Sweep &s) { return s.shape == MMS_STAR ? (size_t)s.nx * s.ny * s.nz * 4 : 0; }

cudaError_t launch_band_tc(const Sweep &s, int path, const CUtensorMap &map, int v, float *scratch)
{
    if (v < 0 || v >= kNumVariants) return cudaErrorInvalidValue;
    if (s.shape == MMS_BOX) return launch_tc<false>(s, path, map, v);
    const int w = 2 * s.r + 1;
    if (is_planar(s.shape)) {
        // Table I's 2D kernels: the planar banded pass straight into the output
        float c2[(2 * kMaxR + 1) * (2 * kMaxR + 1)] = {};
        if (s.shape == MMS_BOX2D) {
            for (int i = 0; i < w * w; ++i) c2[i] = s.coeffs[i];
        } else {
            for (int d = -s.r; d <= s.r; ++d) {
                c2[s.r * w + d + s.r] += s.coeffs[d + s.r];          // x line
                c2[(d + s.r) * w + s.r] += s.coeffs[w + d + s.r];    // y line
            }
        }
        Sweep p = s;
        p.coeffs = c2;
        return launch_tc<true>(p, path, map, v);
    }
    // Star: the in-plane x/y part (with the three centre weights) as a planar
    // banded pass on tensor cores into `scratch` (the paper's temporary buffer
    // for x/y partial results, Sec. 4.3), then the z part on CUDA cores.
    const int r = s.r;
    float c2[(2 * kMaxR + 1) * (2 * kMaxR + 1)] = {};
    for (int d = -r; d <= r; ++d) {
        c2[r * w + d + r] += s.coeffs[0 * w + d + r];  // x line (dy = 0)
        c2[(d + r) * w + r] += s.coeffs[1 * w + d + r];  // y line (dx = 0)
    }
    c2[r * w + r] += s.coeffs[2 * w + r];  // z centre
    Sweep p = s;
    p.coeffs = c2;
    p.out = scratch;
    p.opy = s.nx;
    p.opz = s.nx * s.ny;
    cudaError_t e = launch_tc<true>(p, path, map, v);
    if (e != cudaSuccess) return e;
    switch (r) {
        case 1: return launch_zpass<1>(s, scratch, p.opy, p.opz);
        case 2: return launch_zpass<2>(s, scratch, p.opy, p.opz);
        case 3: return launch_zpass<3>(s, scratch, p.opy, p.opz);
        case 4: return launch_zpass<4>(s, scratch, p.opy, p.opz);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mms
