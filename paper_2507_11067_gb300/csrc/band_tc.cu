// band_tc.cu -- stencil sweeps on the tcgen05 tensor cores.
//
// The paper (Sec. 4.1) turns the 1D stencil along x into a product with a
// banded coefficient matrix, and (Sec. 4.3) a box stencil into 2r+1 shifted
// 1D stencils per plane.  Here the products run on tcgen05 MMAs with the
// grid ROWS on the 128 tensor-memory lanes:
//
//   D[row, (dy, x)] = sum_dz sum_k  A_{z+dz}[row, k] * B_dz[(dy, x), k]
//   out[z][row][x]  = sum_dy D[row + dy, (dy, x)]
//
//  * A, in tensor memory: lane (q, t) = x subtile q (0..3) and input row t
//    (0..31) of one staged plane; it holds the K = 16 input values
//    x0 + q*TXO + k, converted to BF16 (or TF32) hi/lo parts by converter
//    warps that write them with tcgen05.st.  A tile's staged planes form a
//    ring in tensor memory, so the 2r+1 planes of the box are 2r+1 column
//    offsets of the A operand and nothing moves between them;
//  * B, in shared memory (written once per CTA): the band
//    B_dz[(dy, x), k] = c[dz][dy][k - x], zero off the band, for the
//    TXO = 16 - 2r output x positions of a subtile (so K = TXO + 2r = 16
//    exactly, one BF16 MMA step) and the 2r+1 row offsets dy, split into
//    hi/lo parts;
//  * the sum over dy mixes lanes t .. t+2r of one lane quarter: warp
//    shuffles in the epilogue; a quarter holds 32 rows of one subtile, so
//    its TY = 32 - 2r output rows need no other warp's data.
// Split precision (hi*hi + hi*lo + lo*hi into one FP32 accumulator)
// recovers FP32-level accuracy from BF16 or TF32 operands.
//
// Three forms share the kernel:
//  * BOX: the (2r+1)^3 box, 2r+1 planes per output;
//  * PLANAR: a 2D stencil in each plane (Table I's 2D kernels, and the x/y
//    pass of the paper's two-pass star of Sec. 4.3, which writes a
//    temporary grid that star_zpass_kernel completes);
//  * STAR: the 3D star in one pass: the in-plane x and y lines (and the
//    centre) as a 2D band on the output's own plane, the z line added by
//    the converter warps, which see every staged plane anyway and keep the
//    z partial sums of 2r+1 output planes in registers.
//
// Pipeline (persistent CTAs, buffers handed over by mbarriers): warp 0
// stages FP32 plane boxes by TMA; per TMEM lane quarter, one converter warp
// fills the A ring and epilogue warps drain the accumulators and write each
// output subtile with a TMA store; one issuer warp issues every output's
// MMAs in order, converged (the elected lane's MMAs predicated, not branched
// around); after an output's MMAs it commits the release of the A-ring
// slots no later output reads, then the output's accumulator.  A sweep
// whose accumulators and A ring fit in half the TMEM runs two such CTAs per
// SM, whose two workers per lane quarter share converting and draining where
// there are two accumulators (two epilogue warps per quarter and four
// accumulators otherwise, one CTA per SM).
#include <cuda_bf16.h>
#include <stdio.h>

#include "common.cuh"
#include "tc.cuh"

namespace mms {

#ifdef MMS_ROLE_TRACE
// Role trace (debug builds only, -DMMS_ROLE_TRACE): clock cycles that one
// warp of each role in the first eight CTAs spends in its waits and its
// work, summed.
//   [0] producer:  wait staging slot, total
//   [1] issuer 1:  wait planes, wait accumulator, issue, total
//   [2] converter (lane quarter 0): wait staged plane, wait A slot, wait
//                  accumulator (star), conversion and stores, -, total
//   [3] epilogue (quarter 0, even outputs): wait accumulator, loads, reduction
//                  and stores, -, -, -, total
__device__ unsigned long long g_role_trace[4][6];
#define MMS_TRACE_ADD(role, slot, v) \
    do { if (blockIdx.x < 8) atomicAdd(&g_role_trace[role][slot], (unsigned long long)(v)); } while (0)
#define MMS_CLOCK() clock64()
// Timeline of CTA 0 (debug builds only): clock64 stamps of events of its
// first kTl planes / outputs.  Rows: 0 TMA issued (plane), 1 lane quarter 0
// starts converting (plane), 2 ... has its data, 3 ... arrives, 4 issuer
// starts waiting (output), 5 issuer starts issuing, 6 issuer done issuing, 7
// quarter 0's epilogue has the accumulator (output), 8 ... is done, 9, 10,
// 11: lane quarters 1, 2, 3 arrive (plane).
constexpr int kTl = 128;
__device__ unsigned long long g_timeline[12][kTl];
// stamps go to shared memory (tl_smem, after the barriers) and are copied
// out at the end, so that the trace adds no global stores to the roles
#define MMS_TL(row, i) do { if (blockIdx.x == 0 && (i) < kTl) g_timeline[row][i] = clock64(); } while (0)
extern "C" int mms_timeline_read(unsigned long long *host)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;
    return cudaMemcpyFromSymbol(host, g_timeline, sizeof(g_timeline)) != cudaSuccess;
}
extern "C" int mms_role_trace_read(unsigned long long *host, int reset)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;
    if (cudaMemcpyFromSymbol(host, g_role_trace, sizeof(g_role_trace)) != cudaSuccess) return 1;
    if (reset) {
        unsigned long long z[4][6] = {};
        cudaMemcpyToSymbol(g_role_trace, z, sizeof(z));
    }
    return 0;
}
#else
#define MMS_TRACE_ADD(role, slot, v) do { } while (0)
#define MMS_CLOCK() 0ull
#define MMS_TL(row, i) do { } while (0)
#endif

namespace {

enum { P_TF32 = 0, P_3XTF32 = 1, P_BF16X3 = 2 };
enum { M_BOX = 0, M_PLANAR = 1, M_STAR = 2 };

template <int R, int PREC, int MODE>
struct Cfg {
    static constexpr int W = 2 * R + 1;
    static constexpr int WZ = MODE == M_BOX ? W : 1;     // planes whose bands one output multiplies
    static constexpr int RZ = MODE == M_PLANAR ? 0 : R;  // z halo of a tile's staged planes
    static constexpr bool BF = PREC == P_BF16X3;
    static constexpr int K = 16;                         // contraction: input x of one subtile
    // output x per subtile: K - 2r rounded down to a multiple of 4 (12, 12,
    // 8, 8), so that a subtile row of outputs is a 16-byte TMA box row
    static constexpr int TXO = (K - 2 * R) & ~3;
    static constexpr int TX = 4 * TXO;                   // output x per tile (4 subtiles)
    static constexpr int TY = 32 - 2 * R;                // output rows per tile
    static constexpr int NB = W * TXO;                   // band rows (dy, x)
    static constexpr int N = (NB + 15) / 16 * 16;        // MMA N
    static constexpr int ELT = BF ? 2 : 4;               // operand bytes
    static constexpr int KSTEP = BF ? 16 : 8;            // K of one MMA
    static constexpr int NKS = K / KSTEP;                // MMAs per product and plane
    static constexpr int NPARTS = PREC == P_TF32 ? 1 : 2;
    static constexpr int NPROD = PREC == P_TF32 ? 1 : 3;
    static constexpr int ACOLS = K * ELT / 4;            // TMEM columns of one A part
    static constexpr int APL = NPARTS * ACOLS;           // TMEM columns of one staged plane
    static constexpr int ZC = MODE == M_STAR ? (TXO + 15) / 16 * 16 : 0;  // z sums of one output (16-column blocks)
    // A-ring planes needed for progress, with one more converted ahead: the
    // box reads 2r+1 planes per output; a star output reads its centre plane
    // but waits for the plane 2r past its first, which completes its z sum,
    // and a tile's first r (halo) planes are released only with its first
    // output, so 2r+1 planes are resident at a tile's start; planar reads one
    static constexpr int NEED = MODE == M_PLANAR ? 2 : W + 1;
    // Two CTAs per SM where a sweep fits in half the TMEM (its accumulators,
    // z-sum blocks and A ring in 256 columns): two independent pipelines keep
    // the tensor pipe busier than one can.  A dual CTA has ten warps:
    // producer, issuer, and two workers per TMEM lane quarter (a converter
    // and an epilogue warp, or, mixed, two warps that both convert and
    // drain); a single CTA has sixteen: producer, issuer, two idle, and per
    // quarter a converter and two epilogue warps (even and odd outputs).
    // Either way each accumulator slot's laps are waited on in order by one
    // warp.
    static constexpr bool DUAL = N + ZC + NEED * APL <= 256;
    static constexpr int TMEM_COLS = DUAL ? 256 : 512;
    static constexpr int W0 = DUAL ? 2 : 4;              // first worker warp
    static constexpr int ND = DUAL ? (2 * (N + ZC) + NEED * APL <= 256 ? 2 : 1)
                                   : 4 * (N + ZC) + NEED * APL <= 512 ? 4 : 2;
    // TMEM columns: ND accumulators of N | ND z-sum slots of ZC | A ring
    static constexpr int Z0 = ND * N;
    static constexpr int A0 = Z0 + ND * ZC;
    static constexpr int PRF = (TMEM_COLS - A0) / APL < 16 ? (TMEM_COLS - A0) / APL : 16;
    // planes an output reads (or, for the star, waits for) past its first
    static constexpr int OFF_HI = MODE == M_PLANAR ? 0 : 2 * R;
    // Mixed workers (MIX): in a dual CTA with two accumulators, worker wi of
    // a lane quarter converts the planes and drains the outputs of parity
    // wi, so neither sits idle while the other is busy (the star keeps a
    // converter, whose z sums queue in one warp's registers).  Before
    // draining an output a worker converts its planes up to LOOK past the
    // last plane that output reads; the A ring bounds LOOK (a plane's slot
    // is freed once the last output reading the plane PR before it
    // completes), and mixing pays only if the planes of the output two
    // ahead are converted before a drain starts (LOOK >= 2).
    static constexpr int LOOK = (PRF & ~1) - OFF_HI - 1;
    static constexpr bool MIX = DUAL && MODE != M_STAR && ND % 2 == 0 && LOOK >= 2;
    static constexpr int NEPI = DUAL && !MIX ? 1 : 2;    // warps per lane quarter that drain outputs
    static constexpr int PR = MIX ? PRF & ~1 : PRF;      // A ring planes (even when mixed)
    // FP32 staging box: TX + 2r columns (at least), 32 rows, one plane; the
    // row pitch in 16-byte units is odd, so the converters' row reads
    // (8 rows per quarter warp) hit 8 different bank groups
    static constexpr int BOXW = R <= 2 ? 52 : 44;
    static constexpr int STG_BYTES = BOXW * 32 * 4;
    static constexpr int STG_STRIDE = (STG_BYTES + 1023) / 1024 * 1024;
    static constexpr int NST = 8;
    // band: K-major canonical layout, core matrices of 8 rows x 16 bytes,
    // the K chunks of a row group adjacent (LBO = 128 B), row groups SBO apart
    static constexpr int KC = 16 / ELT;                  // K elements per 16-byte chunk
    static constexpr int SBO = K * ELT * 8;
    static constexpr int PART_BYTES = N * K * ELT;
    static constexpr int BAND_BYTES = WZ * NPARTS * PART_BYTES;
    static constexpr int NWARPS = DUAL ? 10 : 16;
    static constexpr int NT = 32 * NWARPS;
    static constexpr size_t OFF_STG = (size_t)(BAND_BYTES + 1023) / 1024 * 1024;
    static constexpr size_t OFF_BAR = OFF_STG + (size_t)NST * STG_STRIDE;
    // Output subtiles staged for TMA stores (one TXO x TY box per epilogue
    // warp and output, two buffers per warp); a subtile row is a 16-byte
    // multiple (TXO % 4 == 0).
    static constexpr bool TSTORE = (TXO * 4) % 16 == 0;
    static constexpr int OBUF = TSTORE ? (TXO * TY * 4 + 127) / 128 * 128 : 0;
    static constexpr size_t OFF_OBUF = OFF_BAR + 1024;
    static constexpr size_t SMEM_NEED = 1024 + OFF_OBUF + 8 * NEPI * (size_t)OBUF;
    // a single CTA takes at least 120 KB, so that two CTAs holding all 512
    // TMEM columns each never share an SM; two dual CTAs fit one SM
    static constexpr size_t SMEM = DUAL ? SMEM_NEED : SMEM_NEED > 120 * 1024 ? SMEM_NEED : 120 * 1024;
    static constexpr bool OK = PR >= NEED && SMEM <= (DUAL ? 113 : 227) * 1024 && A0 + PR * APL <= TMEM_COLS;
    static_assert(OK, "tensor-core configuration does not fit");
    static constexpr uint32_t IDESC = tc::instr_desc(BF ? 1u : 2u, 128, N);
    static_assert(BOXW >= TX - TXO + K && BOXW % 4 == 0 && (BOXW / 4) % 2 == 1, "staging box");
    static_assert(N % 16 == 0 && N <= 256 && (N == 48 || N == 64 || N == 80), "epilogue loads");
    static_assert(2 * NST + 2 * PR + 2 * ND <= 120, "barrier area");
    // TMEM operand and accumulator columns start on 16-column boundaries
    static_assert(Z0 % 16 == 0 && A0 % 16 == 0 && APL % 16 == 0 && N % 16 == 0, "TMEM column alignment");
    static_assert(ND % NEPI == 0, "every epilogue warp owns whole accumulator slots");
    static_assert(!MIX || (PR % 2 == 0 && NST % 2 == 0), "a mixed worker owns the slots of its parity");
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
    int vec;                      // output store width: 4 (float4), 2 (float2) or 1
    int tiles_x, tiles_y, tiles;  // tiles = tiles_x * tiles_y * z chunks
    int nzt;                      // output planes per z chunk
    int zoff;                     // padded input plane of staged plane 0 of chunk 0
    int tstore;                   // outputs leave by TMA stores (the map is valid)
    float cz[2 * kMaxR + 1];      // star: z weights (the centre is in the band)
};

// TMA store of a shared-memory box into a tensor (bulk-group completion),
// and the waits on this thread's bulk groups.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int x, int y, int z)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z), "r"(ptx::smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// every committed group has finished reading its shared-memory source
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed group has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Warp roles: 0 = TMA producer, 1 = MMA issuer (and TMEM owner); then the
// workers, per TMEM lane quarter (warp w reaches lane quarter w % 4) one
// converter and NEPI epilogue warps: warps 4..15 of a single CTA (2 and 3
// idle after set-up), warps 2..9 of a dual one.
template <int R, int PREC, int MODE>
__global__ void __launch_bounds__(Cfg<R, PREC, MODE>::NT, Cfg<R, PREC, MODE>::DUAL ? 2 : 1)
    band_tc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap omap,
                   const __grid_constant__ BoxCoef cf, const __grid_constant__ TcArgs a, unsigned *err)
{
    using C = Cfg<R, PREC, MODE>;
    constexpr int W = C::W;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (ptx::smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *band = smem;
    float *stg = reinterpret_cast<float *>(smem + C::OFF_STG);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    uint64_t *full_stg = bar, *empty_stg = bar + C::NST;
    uint64_t *full_a = empty_stg + C::NST, *empty_a = full_a + C::PR;
    uint64_t *full_d = empty_a + C::PR, *empty_d = full_d + C::ND;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(empty_d + C::ND);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int my_tiles = a.tiles > (int)blockIdx.x ? (a.tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, C::TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < C::NST; ++b) {
            ptx::mbar_init(&full_stg[b], 1);
            ptx::mbar_init(&empty_stg[b], 4);
        }
        for (int b = 0; b < C::PR; ++b) {
            ptx::mbar_init(&full_a[b], 4);
            ptx::mbar_init(&empty_a[b], 1);  // released by the issuer's commit
        }
        for (int b = 0; b < C::ND; ++b) {
            ptx::mbar_init(&full_d[b], 1);
            ptx::mbar_init(&empty_d[b], 4);
        }
        ptx::fence_mbar_init();
        *abort_flag = 0;
    }
    // The band operand: 32-bit word w of the band area holds K element(s)
    // k0 (and k0 + 1 for BF16, high half) of band row n of part p of plane
    // offset dz.
    for (int w = tid; w < C::BAND_BYTES / 4; w += C::NT) {
        const int o = 4 * w;
        const int part = o / C::PART_BYTES, rem = o % C::PART_BYTES;
        const int dzi = part / C::NPARTS, p = part % C::NPARTS;
        const int g = rem / C::SBO, r2 = rem % C::SBO;
        const int jc = r2 / 128, r3 = r2 % 128;
        const int n = g * 8 + r3 / 16;
        const int k0 = jc * C::KC + (r3 % 16) / C::ELT;
        const int dyi = n / C::TXO, xo = n % C::TXO;
        uint32_t word = 0;
#pragma unroll
        for (int h = 0; h < (C::BF ? 2 : 1); ++h) {
            const int d = k0 + h - xo;
            if (n < C::NB && d >= 0 && d <= 2 * R) {
                const float c = MODE == M_BOX ? cf.c[(dzi * W + dyi) * W + d] : cf.c[dyi * W + d];
                word |= split_part<PREC>(c, p) << (16 * h);
            }
        }
        reinterpret_cast<uint32_t *>(band)[w] = word;
    }
    ptx::fence_proxy_async_smem();  // generic writes -> tensor-core reads
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tmem_slot;

    // tile tl of this CTA -> output column origin, first output plane and
    // its number of output planes
    auto tile_of = [&](int tl, int &x0, int &y0, int &z0, int &nzt) {
        const int t = (int)blockIdx.x + tl * (int)gridDim.x;
        const int xt = t % a.tiles_x, yt = (t / a.tiles_x) % a.tiles_y, zc = t / (a.tiles_x * a.tiles_y);
        x0 = xt * C::TX;
        y0 = yt * C::TY;
        z0 = zc * a.nzt;
        nzt = a.nz - z0 < a.nzt ? a.nz - z0 : a.nzt;
    };
    // Bounded wait; on expiry (or once another role has given up) raise the
    // abort flag and return false.
    auto wait = [&](uint64_t *b, uint32_t parity) -> bool {
        if (*abort_flag) return false;
        if (ptx::mbar_wait_bounded(b, parity, err)) return true;
        *abort_flag = 1;
        return false;
    };

    if (warp == 0) {
        // -------------------------------------------------- TMA producer
        const bool leader = ptx::elect_one();
        if (leader) ptx::prefetch_tmap(&tmap);
        int k = 0;  // staged planes issued
        bool ok = true;
        [[maybe_unused]] unsigned long long tw = 0, t00 = MMS_CLOCK();
        for (int tl = 0; tl < my_tiles && ok; ++tl) {
            int x0, y0, z0, nzt;
            tile_of(tl, x0, y0, z0, nzt);
            const int np = nzt + 2 * C::RZ;
            for (int p = 0; p < np; ++p) {
                const int st = k % C::NST;
                [[maybe_unused]] const unsigned long long t0 = MMS_CLOCK();
                ok = __all_sync(0xffffffffu, wait(&empty_stg[st], ((uint32_t)(k / C::NST) & 1u) ^ 1u));
                tw += MMS_CLOCK() - t0;
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                if (leader) {
                    MMS_TL(0, k);
                    ptx::mbar_arrive_expect_tx(&full_stg[st], C::STG_BYTES);
                    ptx::tma_load_3d(stg + (size_t)st * (C::STG_STRIDE / 4), &tmap, x0, y0, z0 + p + a.zoff,
                                     &full_stg[st]);
                }
                __syncwarp();
                ++k;
            }
        }
        if (lane == 0) {
            MMS_TRACE_ADD(0, 0, tw);
            MMS_TRACE_ADD(0, 1, MMS_CLOCK() - t00);
        }
        // every copy this warp issued has landed before the CTA exits
        if (leader)
            for (int st = 0; st < C::NST && st < k; ++st) {
                const int last = (k - 1 - st) / C::NST * C::NST + st;
                ptx::mbar_wait_bounded(&full_stg[st], (uint32_t)(last / C::NST) & 1u, err);
            }
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer
        // One warp issues every output's MMAs in order.  It stays converged:
        // each lane executes the MMA and commit statements, the elected lane
        // alone with its predicate set.  A branch around a single-lane issue
        // costs a reconvergence, and every poll or commit between batches of
        // MMAs leaves the shallow tensor-pipe queue to drain, so the warp
        // waits on each staged plane once, in order (which also keeps it at
        // most one phase behind each A-ring slot), and commits once per
        // output, after the release of the A-ring slots no later output reads.
        const uint32_t on = ptx::elect_one() ? 1u : 0u;
        // planes output z of a tile reads (or, for the star, waits for):
        // up to kb + z + OFF_HI
        const uint64_t bdesc0 = tc::smem_desc(ptx::smem_u32(band), 128, C::SBO);
        int wnext = 0;      // next staged plane to wait on
        int j = 0, kb = 0;  // global output index, global index of the tile's staged plane 0
        int last = -1;      // last output issued
        int rel = 0;        // planes whose A-slot release has been committed (0 .. rel-1)
        bool ok = true;
        [[maybe_unused]] unsigned long long tp = 0, ta = 0, ti = 0, t00 = MMS_CLOCK();
        for (int tl = 0; tl < my_tiles && ok; ++tl) {
            int x0, y0, z0, nzt;
            tile_of(tl, x0, y0, z0, nzt);
            for (int z = 0; z < nzt; ++z, ++j) {
                [[maybe_unused]] const unsigned long long t0 = MMS_CLOCK();
                if (lane == 0) MMS_TL(4, j);
                for (; ok && wnext <= kb + z + C::OFF_HI; ++wnext)
                    ok = __all_sync(0xffffffffu, wait(&full_a[wnext % C::PR], (uint32_t)(wnext / C::PR) & 1u));
                [[maybe_unused]] const unsigned long long t1 = MMS_CLOCK();
                ok = ok && __all_sync(0xffffffffu, wait(&empty_d[j % C::ND], ((uint32_t)(j / C::ND) & 1u) ^ 1u));
                [[maybe_unused]] const unsigned long long t2 = MMS_CLOCK();
                tp += t1 - t0;
                ta += t2 - t1;
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                tc::fence_after_sync();
                if (lane == 0) MMS_TL(5, j);
                // the banded product of each plane the output reads, three
                // split products (one for TF32), into accumulator j % ND; a B
                // descriptor differs from the band's first by a constant added
                // to its start-address field
                const uint32_t dcol = tbase + (uint32_t)((j % C::ND) * C::N);
#pragma unroll
                for (int dzi = 0; dzi < C::WZ; ++dzi) {
                    const int pl = kb + z + (MODE == M_BOX ? dzi : MODE == M_STAR ? R : 0);
                    const uint32_t acol = tbase + (uint32_t)(C::A0 + (pl % C::PR) * C::APL);
#pragma unroll
                    for (int pr = 0; pr < C::NPROD; ++pr) {
                        const int pa = pr == 2 ? 1 : 0;  // data part (A)
                        const int pb = pr == 1 ? 1 : 0;  // band part (B)
#pragma unroll
                        for (int kk = 0; kk < C::NKS; ++kk) {
                            const uint32_t aaddr = acol + (uint32_t)(pa * C::ACOLS + kk * (C::KSTEP * C::ELT / 4));
                            const uint64_t bdesc = bdesc0 + (uint64_t)(((dzi * C::NPARTS + pb) * C::PART_BYTES +
                                                                        kk * (C::KSTEP / C::KC) * 128) >> 4);
                            const uint32_t acc = (dzi | pr | kk) ? 1u : 0u;
                            if constexpr (C::BF)
                                tc::mma_bf16_ts_if(on, dcol, aaddr, bdesc, C::IDESC, acc);
                            else
                                tc::mma_tf32_ts_if(on, dcol, aaddr, bdesc, C::IDESC, acc);
                        }
                    }
                }
                // The A slots of the planes no later output reads are free
                // once these products complete, released here in plane order:
                // the box's plane z is read last by output z, the star's
                // centre plane z+r by output z (its z-halo planes by no
                // product: they go with the tile's first and last outputs),
                // the planar plane z by output z.
                {
                    constexpr int OFF = MODE == M_STAR ? R : 0;
                    if constexpr (MODE == M_STAR)
                        if (z == 0)
                            for (int p = 0; p < R; ++p) tc::mma_commit_if(on, &empty_a[(kb + p) % C::PR]);
                    tc::mma_commit_if(on, &empty_a[(kb + z + OFF) % C::PR]);
                    if constexpr (MODE != M_PLANAR)
                        if (z == nzt - 1)
                            for (int p = nzt + OFF; p < nzt + 2 * R; ++p)
                                tc::mma_commit_if(on, &empty_a[(kb + p) % C::PR]);
                    rel = z == nzt - 1 ? kb + nzt + 2 * C::RZ : kb + z + OFF + 1;
                }
                tc::mma_commit_if(on, &full_d[j % C::ND]);  // accumulator ready for the epilogue
                if (lane == 0) MMS_TL(6, j);
                ti += MMS_CLOCK() - t2;
                last = j;
            }
            kb += nzt + 2 * C::RZ;
        }
        if (lane == 0) {
            MMS_TRACE_ADD(1, 0, tp);
            MMS_TRACE_ADD(1, 1, ta);
            MMS_TRACE_ADD(1, 2, ti);
            MMS_TRACE_ADD(1, 3, MMS_CLOCK() - t00);
        }
        // every MMA issued completes before TMEM is freed
        if (last >= 0) ptx::mbar_wait_bounded(&full_d[last % C::ND], (uint32_t)(last / C::ND) & 1u, err);
        // and every A-slot release committed has arrived before the CTA
        // exits: slot s has had one release per plane s, s + PR, ... < rel
        for (int sl = 0; sl < C::PR; ++sl)
            if (rel > sl) ptx::mbar_wait_bounded(&empty_a[sl], (uint32_t)((rel - 1 - sl) / C::PR) & 1u, err);
    } else if (warp >= C::W0) {
        // ---------------------------------------------------------- workers
        // warp 4 + 4 wi + q: worker wi of TMEM lane quarter q; lane t holds
        // row t of subtile q
        const int q = warp & 3, wi = (warp - C::W0) >> 2, t = lane;
        const uint32_t lane_base = tbase + ((uint32_t)(q * 32) << 16);
        const int ew = C::MIX ? wi : wi - 1;  // this warp's index among its quarter's draining warps
        [[maybe_unused]] float *obuf = reinterpret_cast<float *>(smem + C::OFF_OBUF) +
                                       (size_t)(ew >= 0 ? (ew * 4 + q) * 2 : 0) * (C::OBUF / 4);
        [[maybe_unused]] int nout = 0;  // outputs this epilogue warp has stored
        bool ok = true;
        [[maybe_unused]] unsigned long long ts = 0, ta = 0, td = 0, tc0 = 0, tf = 0, tep = 0, t00 = MMS_CLOCK();

        // Conversion of staged plane k (tile-local p, the tile's outputs
        // start at global index jb): FP32 row -> BF16 (or TF32) hi/lo parts
        // in the A ring; the star also adds the plane's centre values to the
        // z sums of the outputs it reaches (zq: outputs p-2R .. p).
        auto convert = [&](int k, int p, int jb, int nzt, auto &zq) -> bool {
            const int st = k % C::NST, as = k % C::PR;
            [[maybe_unused]] const int zo = p - 2 * R;  // STAR: the output this plane completes
            [[maybe_unused]] const unsigned long long t0 = MMS_CLOCK();
            if (q == 0) MMS_TL(1, k);
            bool good = wait(&full_stg[st], (uint32_t)(k / C::NST) & 1u);
            [[maybe_unused]] const unsigned long long t1 = MMS_CLOCK();
            good = good && wait(&empty_a[as], ((uint32_t)(k / C::PR) & 1u) ^ 1u);
            [[maybe_unused]] const unsigned long long t2 = MMS_CLOCK();
            if constexpr (MODE == M_STAR) {
                const int jo = jb + zo;
                if (zo >= 0 && zo < nzt)
                    good = good && wait(&empty_d[jo % C::ND], ((uint32_t)(jo / C::ND) & 1u) ^ 1u);
            }
            [[maybe_unused]] const unsigned long long t3 = MMS_CLOCK();
            ts += t1 - t0;
            ta += t2 - t1;
            td += t3 - t2;
            if (!__all_sync(0xffffffffu, good)) return false;
            tc::fence_after_sync();  // the slot's last MMAs (and epilogue loads) are ordered before our stores
            if (q == 0) MMS_TL(2, k);
            // the 16 input values of this lane's row
            float v[16];
            const float *row = stg + (size_t)st * (C::STG_STRIDE / 4) + t * C::BOXW + q * C::TXO;
            if constexpr (C::TXO % 4 == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 f = reinterpret_cast<const float4 *>(row)[i];
                    v[4 * i] = f.x; v[4 * i + 1] = f.y; v[4 * i + 2] = f.z; v[4 * i + 3] = f.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float2 f = reinterpret_cast<const float2 *>(row)[i];
                    v[2 * i] = f.x; v[2 * i + 1] = f.y;
                }
            }
            const uint32_t acol = lane_base + (uint32_t)(C::A0 + as * C::APL);
            if constexpr (C::BF) {
                uint32_t hi[8], lo[8];
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    // one cvt packs the pair (even k in the low half)
                    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
                    hi[h] = *reinterpret_cast<const uint32_t *>(&b);
                    const float h0 = __uint_as_float(hi[h] << 16), h1 = __uint_as_float(hi[h] & 0xffff0000u);
                    const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * h] - h0, v[2 * h + 1] - h1);
                    lo[h] = *reinterpret_cast<const uint32_t *>(&l);
                }
                tc::tmem_st_32x32b_x8(acol, hi);
                tc::tmem_st_32x32b_x8(acol + C::ACOLS, lo);
            } else {
                uint32_t hi[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) hi[i] = tf32_rna(v[i]);
                tc::tmem_st_32x32b_x16(acol, hi);
                if constexpr (C::NPARTS == 2) {
                    uint32_t lo[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) lo[i] = tf32_rna(v[i] - __uint_as_float(hi[i]));
                    tc::tmem_st_32x32b_x16(acol + C::ACOLS, lo);
                }
            }
            if constexpr (MODE == M_STAR) {
                // centre values of output row t: input row t + R, from lane t + R
                float cv[C::TXO];
#pragma unroll
                for (int x = 0; x < C::TXO; ++x) cv[x] = __shfl_down_sync(0xffffffffu, v[R + x], R);
                // plane p adds cz[dz] to output p - R - dz = p - 2R + s (s = R - dz)
#pragma unroll
                for (int s = 0; s < W; ++s)
                    if (s != R)
#pragma unroll
                        for (int x = 0; x < C::TXO; ++x) zq[s][x] = fmaf(a.cz[2 * R - s], cv[x], zq[s][x]);
                if (zo >= 0 && zo < nzt) {
                    // output zo is complete: its z sum goes beside its accumulator
                    const uint32_t zcol = lane_base + (uint32_t)(C::Z0 + ((jb + zo) % C::ND) * C::ZC);
#pragma unroll
                    for (int c0 = 0; c0 < C::ZC; c0 += 8) {
                        uint32_t zz[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            zz[i] = c0 + i < C::TXO ? __float_as_uint(zq[0][c0 + i < C::TXO ? c0 + i : 0]) : 0u;
                        tc::tmem_st_32x32b_x8(zcol + c0, zz);
                    }
                }
#pragma unroll
                for (int s = 0; s < W - 1; ++s)
#pragma unroll
                    for (int x = 0; x < C::TXO; ++x) zq[s][x] = zq[s + 1][x];
#pragma unroll
                for (int x = 0; x < C::TXO; ++x) zq[W - 1][x] = 0.f;
            }
            tc::tmem_wait_st();
            tc::fence_before_sync();
            __syncwarp();
            // The staging slot is handed back only now: its values have been
            // consumed (converted and stored), so none of this warp's
            // shared-memory loads can still be in flight when the next TMA
            // copy overwrites the slot.
            if (lane == 0) {
                ptx::mbar_arrive(&empty_stg[st]);
                ptx::mbar_arrive(&full_a[as]);
                MMS_TL(q == 0 ? 3 : 8 + q, k);
            }
            tc0 += MMS_CLOCK() - t3;
            return true;
        };

        // Epilogue of output z of a tile (global index j; the tile's column
        // origin is x0, y0, z0).
        auto epilogue = [&](int j, int z, int x0, int y0, int z0) -> bool {
            const int ds = j % C::ND;
            [[maybe_unused]] const unsigned long long t0 = MMS_CLOCK();
            if (!__all_sync(0xffffffffu, wait(&full_d[ds], (uint32_t)(j / C::ND) & 1u))) return false;
            [[maybe_unused]] const unsigned long long t1 = MMS_CLOCK();
            tf += t1 - t0;
            if (lane == 0 && q == 0) MMS_TL(7, j);
            tc::fence_after_sync();
            uint32_t d[C::N];
            [[maybe_unused]] uint32_t zz[C::ZC > 0 ? C::ZC : 1];
            {
                const uint32_t dc = lane_base + (uint32_t)(ds * C::N);
                [[maybe_unused]] const uint32_t zc = lane_base + (uint32_t)(C::Z0 + ds * C::ZC);
                uint32_t (&d0)[32] = *reinterpret_cast<uint32_t (*)[32]>(&d[0]);
                tc::tmem_ld_32x32b_x32(dc, d0);
                if constexpr (C::N == 48) {
                    uint32_t (&d1)[16] = *reinterpret_cast<uint32_t (*)[16]>(&d[32]);
                    tc::tmem_ld_32x32b_x16(dc + 32, d1);
                } else {
                    uint32_t (&d1)[32] = *reinterpret_cast<uint32_t (*)[32]>(&d[32]);
                    tc::tmem_ld_32x32b_x32(dc + 32, d1);
                    if constexpr (C::N == 80) {
                        uint32_t (&d2)[16] = *reinterpret_cast<uint32_t (*)[16]>(&d[64]);
                        tc::tmem_ld_32x32b_x16(dc + 64, d2);
                    }
                }
                if constexpr (C::ZC == 8) {
                    uint32_t (&z0r)[8] = *reinterpret_cast<uint32_t (*)[8]>(&zz[0]);
                    tc::tmem_ld_32x32b_x8(zc, z0r);
                } else if constexpr (C::ZC == 16) {
                    uint32_t (&z0r)[16] = *reinterpret_cast<uint32_t (*)[16]>(&zz[0]);
                    tc::tmem_ld_32x32b_x16(zc, z0r);
                }
            }
            tc::tmem_wait_ld();
            tc::tmem_regs_ready(d);
            if constexpr (C::ZC > 0) tc::tmem_regs_ready(zz);
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&empty_d[ds]);  // the accumulator is free again
            // out[t][x] = sum_dy D[t + dy][(dy, x)]: lanes t .. t+2R
            float o[C::TXO];
#pragma unroll
            for (int x = 0; x < C::TXO; ++x) {
                float acc = __uint_as_float(d[x]);
#pragma unroll
                for (int dyi = 1; dyi < W; ++dyi)
                    acc += __shfl_down_sync(0xffffffffu, __uint_as_float(d[dyi * C::TXO + x]), dyi);
                if constexpr (MODE == M_STAR) acc += __uint_as_float(zz[x]);
                o[x] = acc;
            }
            const int y = y0 + t, xb = x0 + q * C::TXO, zg = z0 + z;
            if constexpr (C::TSTORE) {
                if (a.tstore) {
                    // the subtile into this warp's buffer for the output's
                    // parity, then one TMA store (clipped at the grid's edges);
                    // the store that last read the buffer is waited for first
                    float *ob = obuf + (size_t)(nout & 1) * (C::OBUF / 4);
                    if (lane == 0) bulk_wait_read_all();
                    __syncwarp();
                    if (t < C::TY) {
#pragma unroll
                        for (int i = 0; i < C::TXO / 4; ++i)
                            reinterpret_cast<float4 *>(ob + t * C::TXO)[i] =
                                make_float4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
                    }
                    ptx::fence_proxy_async_smem();  // generic writes -> the TMA unit's reads
                    __syncwarp();
                    if (lane == 0 && xb < a.nx) {
                        tma_store_3d(&omap, ob, xb, y0, zg);
                        bulk_commit();
                    }
                    ++nout;
                    if (lane == 0 && q == 0) MMS_TL(8, j);
                    tep += MMS_CLOCK() - t1;
                    return true;
                }
            }
            if (t < C::TY && y < a.ny && xb < a.nx) {
                float *op = a.out + (int64_t)zg * a.opz + (int64_t)y * a.opy + xb;
                const bool full = xb + C::TXO <= a.nx;
                if (C::TXO % 4 == 0 && full && a.vec == 4) {
#pragma unroll
                    for (int i = 0; i < C::TXO / 4; ++i)
                        reinterpret_cast<float4 *>(op)[i] = make_float4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
                } else if (full && a.vec >= 2) {
#pragma unroll
                    for (int i = 0; i < C::TXO / 2; ++i)
                        reinterpret_cast<float2 *>(op)[i] = make_float2(o[2 * i], o[2 * i + 1]);
                } else {
#pragma unroll
                    for (int x = 0; x < C::TXO; ++x)
                        if (xb + x < a.nx) op[x] = o[x];
                }
            }
            if (lane == 0 && q == 0) MMS_TL(8, j);
            tep += MMS_CLOCK() - t1;
            return true;
        };

        if constexpr (C::MIX) {
            // Worker wi converts the planes and drains the outputs of parity
            // wi (global indices; a tile's plane and output indices share
            // their parity, 2r being even), interleaved: before draining an
            // output it converts its planes up to LOOK past the last plane
            // that output reads.  Rank the conversion of plane k at k - LOOK
            // and the drain of output j at (the last plane j reads) + 1/2:
            // every worker's sequence is in rank order, and every wait is on
            // an item of lower rank -- a drain on its output's planes and on
            // the drain of its accumulator slot's previous output, a
            // conversion on the planes before it in the staging ring and on
            // the products that free its A slot, which read no plane past
            // k - PR + OFF_HI, with PR > OFF_HI + LOOK -- so no wait closes a
            // cycle.
            float zq[1][1];
            // plane cursor: global plane kc of tile tp (first plane kbp,
            // first output jbp, nzp outputs)
            int kc = wi, tp = 0, kbp = 0, jbp = 0, nzp = 0, xd, yd, zd;
            bool planes_left = my_tiles > 0;
            if (planes_left) tile_of(0, xd, yd, zd, nzp);
            auto plane_fix = [&]() {
                while (planes_left && kc - kbp >= nzp + 2 * C::RZ) {
                    kbp += nzp + 2 * C::RZ;
                    jbp += nzp;
                    if (++tp >= my_tiles) planes_left = false;
                    else tile_of(tp, xd, yd, zd, nzp);
                }
            };
            plane_fix();
            // output cursor: global output jd of tile to (first plane kbo,
            // first output jbo, its origin and nzo outputs)
            int jd = wi, to = 0, kbo = 0, jbo = 0, nzo = 0, x0o = 0, y0o = 0, z0o = 0;
            bool outs_left = my_tiles > 0;
            if (outs_left) tile_of(0, x0o, y0o, z0o, nzo);
            auto out_fix = [&]() {
                while (outs_left && jd - jbo >= nzo) {
                    kbo += nzo + 2 * C::RZ;
                    jbo += nzo;
                    if (++to >= my_tiles) outs_left = false;
                    else tile_of(to, x0o, y0o, z0o, nzo);
                }
            };
            out_fix();
            while (ok && (planes_left || outs_left)) {
                // the last plane the next output of this parity reads
                const int need = outs_left ? kbo + (jd - jbo) + C::OFF_HI : 0;
                if (planes_left && (!outs_left || kc <= need + C::LOOK)) {
                    ok = convert(kc, kc - kbp, jbp, nzp, zq);
                    kc += 2;
                    plane_fix();
                } else {
                    ok = epilogue(jd, jd - jbo, x0o, y0o, z0o);
                    jd += 2;
                    out_fix();
                }
            }
            if constexpr (C::TSTORE)
                if (lane == 0) bulk_wait_all();
        } else if (wi == 0) {
            // every staged plane in order (the star's z sums in registers)
            float zq[MODE == M_STAR ? W : 1][MODE == M_STAR ? C::TXO : 1];
            int k = 0, jb = 0;
            for (int tl = 0; tl < my_tiles && ok; ++tl) {
                int x0, y0, z0, nzt;
                tile_of(tl, x0, y0, z0, nzt);
                if constexpr (MODE == M_STAR) {
#pragma unroll
                    for (int s2 = 0; s2 < W; ++s2)
#pragma unroll
                        for (int x = 0; x < C::TXO; ++x) zq[s2][x] = 0.f;
                }
                for (int p = 0; p < nzt + 2 * C::RZ && ok; ++p, ++k) ok = convert(k, p, jb, nzt, zq);
                jb += nzt;
            }
        } else {
            // the epilogues of the even (worker 1) or odd (worker 2) outputs
            int j = 0;
            for (int tl = 0; tl < my_tiles && ok; ++tl) {
                int x0, y0, z0, nzt;
                tile_of(tl, x0, y0, z0, nzt);
                for (int z = 0; z < nzt && ok; ++z, ++j)
                    if (j % C::NEPI == wi - 1) ok = epilogue(j, z, x0, y0, z0);
            }
            // this warp's output stores are complete (and their sources
            // read) before the CTA exits
            if constexpr (C::TSTORE)
                if (lane == 0) bulk_wait_all();
        }
        if (!ok) *abort_flag = 1;
        if (lane == 0 && warp == 4) {
            MMS_TRACE_ADD(2, 0, ts);
            MMS_TRACE_ADD(2, 1, ta);
            MMS_TRACE_ADD(2, 2, td);
            MMS_TRACE_ADD(2, 3, tc0);
            MMS_TRACE_ADD(2, 5, MMS_CLOCK() - t00);
        }
        if (lane == 0 && warp == 8) {
            MMS_TRACE_ADD(3, 0, tf);
            MMS_TRACE_ADD(3, 1, tep);
            MMS_TRACE_ADD(3, 5, MMS_CLOCK() - t00);
        }
    }

    __syncwarp();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, C::TMEM_COLS);
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

// What one launch computes: the band weights (box: (2r+1)^3; planar and
// star: the (2r+1)^2 in-plane set), the star's z weights, where the staged
// planes start, and where the results go.
struct Launch {
    const float *band;
    const float *cz;   // star only
    int zoff;
    float *out;
    int64_t opy, opz;
};

template <int R, int PREC, int MODE>
cudaError_t launch_r(const Sweep &s, const CUtensorMap &map, int nzt, const Launch &L)
{
    using C = Cfg<R, PREC, MODE>;
    static_assert(C::OK, "tensor-core configuration does not fit");
    BoxCoef cf{};
    const int ncoef = MODE == M_BOX ? C::W * C::W * C::W : C::W * C::W;
    for (int i = 0; i < ncoef; ++i) cf.c[i] = L.band[i];
    TcArgs a{};
    a.out = L.out;
    a.opy = L.opy;
    a.opz = L.opz;
    a.nx = (int)s.nx;
    a.ny = (int)s.ny;
    a.nz = (int)s.nz;
    const uintptr_t ob = reinterpret_cast<uintptr_t>(L.out);
    a.vec = (L.opy % 4 == 0 && L.opz % 4 == 0 && ob % 16 == 0) ? 4 : (L.opy % 2 == 0 && L.opz % 2 == 0 && ob % 8 == 0) ? 2 : 1;
    const int64_t tx = (s.nx + C::TX - 1) / C::TX, ty = (s.ny + C::TY - 1) / C::TY, tz = (s.nz + nzt - 1) / nzt;
    if (tx * ty * tz > (int64_t)1 << 30) return cudaErrorInvalidValue;
    a.tiles_x = (int)tx;
    a.tiles_y = (int)ty;
    a.tiles = (int)(tx * ty * tz);
    a.nzt = nzt;
    a.zoff = L.zoff;
    if (MODE == M_STAR)
        for (int d = 0; d < C::W; ++d) a.cz[d] = L.cz[d];
    // outputs by TMA stores where the subtile rows and the output's pitches
    // are 16-byte multiples (and the map encodes); else from registers
    CUtensorMap omap{};
    a.tstore = C::TSTORE && a.vec == 4 &&
               encode_tmap_3d(&omap, L.out, s.nx, s.ny, s.nz, L.opy, L.opz, C::TSTORE ? C::TXO : 4, C::TY, 1);
    auto kern = band_tc_kernel<R, PREC, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    // persistent: one CTA per SM, two for the dual configuration
    const int slots = num_sms() * (C::DUAL ? 2 : 1);
    const int grid = a.tiles < slots ? a.tiles : slots;
    kern<<<grid, C::NT, C::SMEM, s.stream>>>(map, omap, cf, a, device_error_word());
    return cudaGetLastError();
}

// Variants: output planes per z chunk of a tile (52 and 40 split 512
// planes into 10 and 13 chunks, whose tiles spread more evenly over the
// persistent CTAs than 8 or 16 chunks; the autotuner weighs that against
// the halo planes each chunk restages); the star's variants kNumTile.. run
// the paper's two-pass form (x/y pass into a temporary grid, then the z
// pass).
constexpr int kNzt[] = {64, 32, 128, 16, 52, 40};
constexpr int kNumTile = sizeof(kNzt) / sizeof(int);

template <int PREC, int MODE>
cudaError_t launch_mode(const Sweep &s, const CUtensorMap &map, int nzt, const Launch &L)
{
    switch (s.r) {
        case 1: return launch_r<1, PREC, MODE>(s, map, nzt, L);
        case 2: return launch_r<2, PREC, MODE>(s, map, nzt, L);
        case 3: return launch_r<3, PREC, MODE>(s, map, nzt, L);
        case 4: return launch_r<4, PREC, MODE>(s, map, nzt, L);
        default: return cudaErrorInvalidValue;
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

template <int MODE>
cudaError_t launch_prec(const Sweep &s, int path, const CUtensorMap &map, int nzt, const Launch &L)
{
    switch (prec_of(path)) {
        case P_TF32: return launch_mode<P_TF32, MODE>(s, map, nzt, L);
        case P_3XTF32: return launch_mode<P_3XTF32, MODE>(s, map, nzt, L);
        case P_BF16X3: return launch_mode<P_BF16X3, MODE>(s, map, nzt, L);
        default: return cudaErrorInvalidValue;
    }
}

// z part of the two-pass star after the tensor-core x/y pass:
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

// The in-plane (2r+1)^2 weights [dy][dx] of a star (x line, y line and the
// centre weights) or of a planar shape.
void planar_weights(const Sweep &s, bool with_z_centre, float *c2)
{
    const int r = s.r, w = 2 * r + 1;
    for (int i = 0; i < w * w; ++i) c2[i] = 0.f;
    if (s.shape == MMS_BOX2D) {
        for (int i = 0; i < w * w; ++i) c2[i] = s.coeffs[i];
        return;
    }
    for (int d = -r; d <= r; ++d) {
        c2[r * w + d + r] += s.coeffs[d + r];          // x line (dy = 0)
        c2[(d + r) * w + r] += s.coeffs[w + d + r];    // y line (dx = 0)
    }
    if (with_z_centre) c2[r * w + r] += s.coeffs[2 * w + r];
}

// The pipeline constants of one configuration, for mms_tc_pipeline_config.
template <int R, int PREC, int MODE>
int pipeline_config(int32_t *cfg, int n)
{
    using C = Cfg<R, PREC, MODE>;
    const int32_t v[] = {C::MIX ? 1 : 0, C::LOOK, C::PR, C::NST, C::ND, C::OFF_HI, C::RZ, C::DUAL ? 1 : 0, C::NEPI};
    constexpr int nv = sizeof(v) / sizeof(v[0]);
    for (int i = 0; i < nv && i < n; ++i) cfg[i] = v[i];
    return nv;
}

template <int PREC, int MODE>
int pipeline_config_r(int r, int32_t *cfg, int n)
{
    switch (r) {
        case 1: return pipeline_config<1, PREC, MODE>(cfg, n);
        case 2: return pipeline_config<2, PREC, MODE>(cfg, n);
        case 3: return pipeline_config<3, PREC, MODE>(cfg, n);
        case 4: return pipeline_config<4, PREC, MODE>(cfg, n);
        default: return -1;
    }
}

template <int MODE>
int pipeline_config_p(int prec, int r, int32_t *cfg, int n)
{
    switch (prec) {
        case P_TF32: return pipeline_config_r<P_TF32, MODE>(r, cfg, n);
        case P_3XTF32: return pipeline_config_r<P_3XTF32, MODE>(r, cfg, n);
        case P_BF16X3: return pipeline_config_r<P_BF16X3, MODE>(r, cfg, n);
        default: return -1;
    }
}

}  // namespace

int band_tc_supported(int shape, int r, int path)
{
    return shape >= MMS_STAR && shape <= MMS_BOX2D && r >= 1 && r <= kMaxR && prec_of(path) >= 0;
}

int band_tc_variants(int shape, int r, int path)
{
    if (!band_tc_supported(shape, r, path)) return 0;
    return shape == MMS_STAR ? 2 * kNumTile : kNumTile;
}

int band_tc_two_pass(int shape, int v) { return shape == MMS_STAR && v >= kNumTile && v < 2 * kNumTile; }

int band_tc_two_pass_variant(int v) { return kNumTile + (v >= 0 ? v % kNumTile : 0); }

void band_tc_box(int shape, int r, int path, int v, int *bx, int *by, int *bz, int *swz)
{
    (void)shape; (void)path; (void)v;
    // the kernel's own staging width (it does not depend on precision or form)
    static const int boxw[kMaxR + 1] = {0, Cfg<1, P_BF16X3, M_BOX>::BOXW, Cfg<2, P_BF16X3, M_BOX>::BOXW,
                                        Cfg<3, P_BF16X3, M_BOX>::BOXW, Cfg<4, P_BF16X3, M_BOX>::BOXW};
    *bx = r >= 1 && r <= kMaxR ? boxw[r] : 0;
    *by = 32;
    *bz = 1;
    *swz = 0;
}

size_t band_tc_scratch_bytes(const Sweep &s)
{
    return band_tc_two_pass(s.shape, s.variant) ? (size_t)s.nx * s.ny * s.nz * 4 : 0;
}

cudaError_t launch_band_tc(const Sweep &s, int path, const CUtensorMap &map, int v, float *scratch)
{
    if (v < 0 || v >= band_tc_variants(s.shape, s.r, path)) return cudaErrorInvalidValue;
    const int nzt = kNzt[v % kNumTile];
    const int w = 2 * s.r + 1;
    float c2[(2 * kMaxR + 1) * (2 * kMaxR + 1)];
    if (s.shape == MMS_BOX) {
        const Launch L{s.coeffs, nullptr, 0, s.out, s.opy, s.opz};
        return launch_prec<M_BOX>(s, path, map, nzt, L);
    }
    if (is_planar(s.shape)) {
        // Table I's 2D kernels: the planar banded pass straight into the output
        planar_weights(s, false, c2);
        const Launch L{c2, nullptr, 0, s.out, s.opy, s.opz};
        return launch_prec<M_PLANAR>(s, path, map, nzt, L);
    }
    if (!band_tc_two_pass(s.shape, v)) {
        // the star in one pass: x/y lines and the centre on tensor cores, the
        // z line summed by the converter warps
        planar_weights(s, true, c2);
        const Launch L{c2, s.coeffs + 2 * w, 0, s.out, s.opy, s.opz};
        return launch_prec<M_STAR>(s, path, map, nzt, L);
    }
    // The paper's two-pass star (Sec. 4.3): the in-plane x/y part with the
    // three centre weights into `scratch` (its temporary buffer), then the z
    // part on CUDA cores.
    if (!scratch) return cudaErrorInvalidValue;
    planar_weights(s, true, c2);
    const Launch L{c2, nullptr, s.r, scratch, s.nx, s.nx * s.ny};
    cudaError_t e = launch_prec<M_PLANAR>(s, path, map, nzt, L);
    if (e != cudaSuccess) return e;
    switch (s.r) {
        case 1: return launch_zpass<1>(s, scratch, s.nx, s.nx * s.ny);
        case 2: return launch_zpass<2>(s, scratch, s.nx, s.nx * s.ny);
        case 3: return launch_zpass<3>(s, scratch, s.nx, s.nx * s.ny);
        case 4: return launch_zpass<4>(s, scratch, s.nx, s.nx * s.ny);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mms

extern "C" int32_t mms_tc_pipeline_config(int32_t shape, int32_t radius, int32_t path, int32_t *cfg, int32_t ncfg)
{
    using namespace mms;
    if (ncfg < 0 || (ncfg > 0 && !cfg) || !band_tc_supported(shape, radius, path)) return -1;
    const int prec = prec_of(path);
    if (shape == MMS_BOX) return pipeline_config_p<M_BOX>(prec, radius, cfg, ncfg);
    if (shape == MMS_STAR) return pipeline_config_p<M_STAR>(prec, radius, cfg, ncfg);
    return pipeline_config_p<M_PLANAR>(prec, radius, cfg, ncfg);
}
