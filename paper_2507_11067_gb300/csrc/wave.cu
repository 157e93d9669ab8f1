// wave.cu -- fused acoustic wave step, its discrete adjoint, and the small
// pointwise kernels around them (model, chain rule, FP64 dot product).
//
// The forward kernel is the star sweep of sweep_cc.cu with the leapfrog
// update fused into its epilogue: the Laplacian of a^n never leaves
// registers, so one step moves 16 bytes per point (read a^n, a^{n-1}, m;
// write a^{n+1}) plus the L2-served halos.  Shots are independent and run
// as separate grid slices of the same launch.
//
// The adjoint kernel computes, per point and shot,
//   lam^n = R^T r^n + 2 g lam^{n+1} + L(m g lam^{n+1}) - g^2 lam^{n+2}
//   grad += g lam^{n+1} (L a^n)     (FP64, all shots)
// staging lam^{n+1}, m and a^n planes with TMA; the stencil input
// q = m g lam^{n+1} is formed plane by plane in shared memory.
//
// The gradient path runs the same recursion in the scaled variable
// mu = m g lam (pointwise).  Multiplying the update by m g at the output
// point gives
//   mu^n = g (2 mu^{n+1} + m L mu^{n+1} - g mu^{n+2} + m R^T r^n)
//   grad += mu^{n+1} (L a^n)          (= m times the lam-form term)
// -- the forward step's form (the stencil on the state itself, m and g after
// it) -- so it runs on the forward kernel with no per-plane product and
// no barrier between forming and reading it; the accumulated gradient is
// divided by m once at the end (divide_m_kernel).  It needs m > 0.
#include "common.cuh"
#include "tile.cuh"
#include "wave.cuh"

namespace mms {

__device__ unsigned g_error_word = 0;

unsigned *device_error_word()
{
    static unsigned *addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_error_word) != cudaSuccess) return nullptr;
        addr[dev] = static_cast<unsigned *>(p);
    }
    return addr[dev];
}

namespace {

// Failure-path self-test: one CTA waits, bounded by limit_ns, on an mbarrier
// phase that nothing completes; the wait runs out, records the timeout in
// the error word and the kernel returns -- the path that every bounded wait
// of the library takes, exercised without a fault.
__global__ void wait_selftest_kernel(unsigned long long limit_ns, unsigned *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    (void)ptx::mbar_wait_bounded(&bar, 0, err, limit_ns);
}

// FP32 -> FP64 by the IEEE-754 layouts (sign kept, exponent rebased by
// 1023 - 127, fraction shifted up 29 bits), on the integer units: GB300's
// FP64 pipe issues about two instructions per clock per SM, which a
// conversion per point and plane would saturate.  Exact for every FP32
// value: a denormal f (fraction field F, f = F 2^-149) is normalised by the
// position of F's leading one (FP64 reaches far below 2^-149).
__device__ __forceinline__ double widen(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu, frac = u & 0x7fffffu;
    uint64_t d = (uint64_t)(u & 0x80000000u) << 32;
    if (e == 0xffu) {
        d |= (uint64_t)0x7ffu << 52 | (uint64_t)frac << 29;
    } else if (e != 0u) {
        d |= (uint64_t)(e + 896u) << 52 | (uint64_t)frac << 29;
    } else if (frac != 0u) {
        // leading one of F at bit b = 23 - s: f = 1.xxx 2^(-126 - s)
        const uint32_t sh = (uint32_t)__clz(frac) - 8u;
        d |= (uint64_t)(897u - sh) << 52 | (uint64_t)((frac << sh) & 0x7fffffu) << 29;
    }
    return __longlong_as_double((long long)d);
}

// Ring stage s: [a^n plane + halo | m tile | a^{n-1} tile | a^n tile].  The
// interior tiles of output plane zo = j - 2R (m, a^{n-1} and the centre
// values of a^n) ride in the stage of input plane j, the plane that completes
// zo, so every operand arrives asynchronously and no register queue of
// centre values is needed.
// The kernel's three forms: the forward step; the forward step that also
// writes L a^n; the adjoint step in the scaled variable mu = m G lam, whose
// update has the forward step's form (the stencil acts on the state itself),
// with the receiver residual m r^n in place of the source and the FP64
// gradient term mu^{n+1} (L a^n) = m G lam^{n+1} (L a^n), L a^n read from a
// fifth tile.
enum { K_FWD = 0, K_FWD_LAP = 1, K_ADJ_SCALED = 2 };

template <int R, int TX, int TY, int PY, int S, int MODE = K_FWD>
struct FwdGeom {
    using G = Geom<R, TX, TY, PY, S>;
    using I = Interior<R, TX>;
    static constexpr int MT = I::BXI * TY;                  // floats of one interior tile
    // sub-tile offsets rounded to 32 floats: every TMA destination is 128-byte aligned
    static constexpr int OFF_M = (G::PLANE + 31) & ~31;
    static constexpr int OFF_P = OFF_M + ((MT + 31) & ~31);
    static constexpr int OFF_C = OFF_P + ((MT + 31) & ~31);
    static constexpr int OFF_L = OFF_C + ((MT + 31) & ~31);  // adjoint: L a^n
    static constexpr int STAGE = OFF_L + (MODE == K_ADJ_SCALED ? ((MT + 31) & ~31) : 0);
    // adjoint: two FP64 buffers of an output plane's gradient terms (TY x
    // TX), 128-byte aligned after the ring's barriers and abort flag
    static constexpr size_t OFF_GB = ((size_t)S * STAGE * 4 + S * sizeof(uint64_t) + 16 + 127) / 128 * 128;
    static constexpr size_t GB_BYTES = MODE == K_ADJ_SCALED ? 2 * (size_t)TY * TX * sizeof(double) : 0;
    static constexpr size_t SMEM = 128 + OFF_GB + GB_BYTES;
};

// Programmatic dependent launch: the next kernel of the stream (launched
// with the programmatic-serialization attribute) may start once every CTA
// of this grid has signalled; a kernel so launched waits, before it touches
// global memory another kernel wrote or reads, until the previous grid has
// completed and its writes are visible.  Both are no-ops without the
// attribute.
__device__ __forceinline__ void launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launches a kernel whose prologue may overlap the previous kernel of the
// stream (programmatic stream serialization); the kernel calls
// wait_prior_grid() before its first dependent global access.  A stream
// being captured into a graph gets a plain launch (a replayed graph has no
// launch gaps to hide).
template <typename... KArgs, typename... Args>
cudaError_t launch_overlapped(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusNone;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = cs == cudaStreamCaptureStatusNone ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

// Bulk reduction of an FP64 row from shared memory into global memory (the
// L2 adds it), in this thread's bulk groups; addresses 16-byte aligned, size
// a multiple of 16 bytes.
__device__ __forceinline__ void bulk_add_f64(double *dst, const double *src, uint32_t bytes)
{
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;" ::"l"(dst),
                 "r"(ptx::smem_u32(src)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most the most recent group may still be reading its source
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Operands of the scaled adjoint (unused by the forward forms).
struct AdjArgs {
    const float *resid;  // nshots*ny*nx on the receiver plane, or null
    double *grad;        // FP64 gradient, or null (no gradient term, tlap unused)
    int gvec;            // rows of four doubles 32-byte aligned
    int gbulk;           // one shared slice, nx even, grad 16-byte aligned: rows added by bulk reductions
};

template <int R, int TX, int TY, int PY, int S, int MODE>
__global__ void __launch_bounds__(Geom<R, TX, TY, PY, S>::NT)
    wave_fwd_kernel(const __grid_constant__ CUtensorMap tcur, const __grid_constant__ CUtensorMap tm,
                    const __grid_constant__ CUtensorMap tprev, const __grid_constant__ CUtensorMap tctr,
                    const __grid_constant__ CUtensorMap tlap, const __grid_constant__ StarCoef cf,
                    const __grid_constant__ WaveGeo geo, float *__restrict__ pnext,
                    const float *__restrict__ amp, float *__restrict__ rec, float *__restrict__ lapout,
                    const __grid_constant__ AdjArgs adj, int tz, int nzc, int vec, unsigned *err)
{
    constexpr bool LAPOUT = MODE == K_FWD_LAP;
    constexpr bool ADJ = MODE == K_ADJ_SCALED;
    using G = Geom<R, TX, TY, PY, S>;
    using F = FwdGeom<R, TX, TY, PY, S, MODE>;
    using I = Interior<R, TX>;
    constexpr int W = G::W;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_align128(smem_raw);
    float *stages = reinterpret_cast<float *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)S * F::STAGE * sizeof(float));
    int &abort_flag = *reinterpret_cast<int *>(full + S);

    // the next step's kernel may set up while this one runs
    launch_dependents();
    const int tid = threadIdx.x;
    const int tx = tid % G::NTX, ty = tid / G::NTX;
    // The adjoint's shots of one z chunk are adjacent in launch order, so
    // that they run together and their FP64 gradient rows meet in L2 (its
    // z chunks can span several waves); the forward forms keep a shot's
    // chunks adjacent (measured faster for them: 8 x 512^3, 2.97 against
    // 3.25 ms per step).
    const int sh = ADJ ? blockIdx.z % geo.nshots : blockIdx.z / nzc;
    const int zc = ADJ ? blockIdx.z / geo.nshots : blockIdx.z % nzc;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, zb = zc * tz;
    const int nzt = min(tz, geo.nz - zb);
    const int P = nzt + 2 * R;
    const int ry0 = ty * PY;
    const int gx = x0 + 4 * tx;
    const int sx = ADJ ? -1 : geo.src[sh][0], sy = ADJ ? -1 : geo.src[sh][1], sz = ADJ ? -1 : geo.src[sh][2];
    const bool has_grad = ADJ && adj.grad != nullptr;
    // The shots' terms go to one shared gradient: each output plane's terms
    // are gathered in shared memory and each row is added by one bulk
    // reduction (the L2 does the adds), instead of one FP64 atomic per point.
    [[maybe_unused]] const bool gbulk = has_grad && geo.gss == 0 && adj.gbulk;
    [[maybe_unused]] double *gbuf = reinterpret_cast<double *>(smem + F::OFF_GB);
    const int ntiles = has_grad ? 4 : 3;

    auto issue = [&](int j, int s) {
        float *st = stages + (size_t)s * F::STAGE;
        const bool inner = j >= 2 * R;  // this plane completes output plane j - 2R
        ptx::mbar_arrive_expect_tx(&full[s], (G::PLANE + (inner ? ntiles * F::MT : 0)) * sizeof(float));
        ptx::tma_load_4d(st, &tcur, x0, y0, zb + j, sh, &full[s]);
        if (inner) {
            const int zp = zb + j - R;  // padded plane of output zo = j - 2R
            const int xs = x0 + (R & ~3);
            ptx::tma_load_3d(st + F::OFF_M, &tm, xs, y0 + R, zp, &full[s]);
            ptx::tma_load_4d(st + F::OFF_P, &tprev, xs, y0 + R, zp, sh, &full[s]);
            ptx::tma_load_4d(st + F::OFF_C, &tctr, xs, y0 + R, zp, sh, &full[s]);
            if (has_grad) ptx::tma_load_4d(st + F::OFF_L, &tlap, xs, y0 + R, zp, sh, &full[s]);
        }
    };
    if (tid == 0) {
        ptx::prefetch_tmap(&tcur);
        ptx::prefetch_tmap(&tm);
        ptx::prefetch_tmap(&tprev);
        ptx::prefetch_tmap(&tctr);
        if (has_grad) ptx::prefetch_tmap(&tlap);
#pragma unroll
        for (int s = 0; s < S; ++s) ptx::mbar_init(&full[s], 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
    }
    // the previous step's fields are complete before any is read or written
    wait_prior_grid();
    __syncthreads();
    if (tid == 0)
        for (int j = 0; j < S && j < P; ++j) issue(j, j);
    float gxs[4], gys[PY];
#pragma unroll
    for (int k = 0; k < 4; ++k) gxs[k] = sponge(gx + k, geo.nx, geo.sponge_w, geo.sponge_a);
#pragma unroll
    for (int i = 0; i < PY; ++i) gys[i] = sponge(y0 + ry0 + i, geo.ny, geo.sponge_w, geo.sponge_a);

    float acc[W][PY][4];
#pragma unroll
    for (int kk = 0; kk < W; ++kk)
#pragma unroll
        for (int i = 0; i < PY; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[kk][i][k] = 0.f;

    const float samp = ADJ ? 0.f : amp[sh];
    const int64_t shot_off = (int64_t)sh * geo.ss;
    for (int j = 0; j < P; ++j) {
        const int s = j % S;
        const float *st = stages + (size_t)s * F::STAGE;
        const int zo = j - 2 * R;  // output plane completed by plane j
        float mv[PY][4], pv[PY][4], cv[PY][4];
        [[maybe_unused]] float lv[PY][4];
        if (ptx::mbar_wait_bounded(&full[s], (uint32_t)(j / S) & 1u, err)) {
            float unused[PY][4];
            star_plane<R, PY, G::BX, G::NV>(st, cf, acc, unused, tx, ry0);
            if (zo >= 0) {
#pragma unroll
                for (int i = 0; i < PY; ++i) {
                    // interior tiles: row ry0+i, columns 4tx+OFF .. +3
                    load_center<I::OFF>(st + F::OFF_M + (ry0 + i) * I::BXI + 4 * tx, mv[i]);
                    load_center<I::OFF>(st + F::OFF_P + (ry0 + i) * I::BXI + 4 * tx, pv[i]);
                    load_center<I::OFF>(st + F::OFF_C + (ry0 + i) * I::BXI + 4 * tx, cv[i]);
                    if constexpr (ADJ)
                        if (has_grad) load_center<I::OFF>(st + F::OFF_L + (ry0 + i) * I::BXI + 4 * tx, lv[i]);
                }
            }
        } else {
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) {
            if constexpr (ADJ) bulk_wait_all();  // no reduction still reads this CTA's buffers
            return;
        }
        if (tid == 0 && j + S < P) issue(j + S, s);
        if (zo >= 0) {
            const int z = zb + zo;
            const float gzv = sponge(z, geo.nz, geo.sponge_w, geo.sponge_a);
            // this output plane's gradient buffer; the reductions of the plane
            // before last, which read it, are done first
            [[maybe_unused]] double *gb = gbuf + (size_t)(zo & 1) * (TY * TX);
            if constexpr (ADJ) {
                if (gbulk) {
                    if (tx == 0) bulk_wait_read_1();
                    __syncwarp();
                }
            }
#pragma unroll
            for (int i = 0; i < PY; ++i) {
                const int y = y0 + ry0 + i;
                if (y >= geo.ny || gx >= geo.nx) continue;
                const int64_t mp = (int64_t)(z + R) * geo.pz + (int64_t)(y + R) * geo.py + (gx + R);
                float *pp = pnext + shot_off + mp;
                float res[4];
                [[maybe_unused]] double gd[4] = {0.0, 0.0, 0.0, 0.0};
                [[maybe_unused]] const bool at_rec = ADJ && adj.resid && z == geo.rec_z;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float g = gxs[k] * gys[i] * gzv;
                    float v = 2.f * cv[i][k] + mv[i][k] * acc[0][i][k] - g * pv[i][k];
                    if constexpr (ADJ) {
                        if (at_rec && gx + k < geo.nx)
                            v += mv[i][k] * adj.resid[((int64_t)sh * geo.ny + y) * geo.nx + gx + k];
                        // mu^{n+1} (L a^n) = m G lam^{n+1} (L a^n): m is the same
                        // at every step, so the sum is divided by it once, at
                        // the end (mms_grad_divide_m).  The term in FP32 (its
                        // operands are FP32), accumulated in FP64.
                        if (has_grad) gd[k] = widen(cv[i][k] * lv[i][k]);
                    } else {
                        if (gx + k == sx && y == sy && z == sz) v += samp;
                    }
                    res[k] = g * v;
                }
                if (vec && gx + 3 < geo.nx) {
                    *reinterpret_cast<float4 *>(pp) = make_float4(res[0], res[1], res[2], res[3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (gx + k < geo.nx) pp[k] = res[k];
                }
                if constexpr (LAPOUT) {  // L a^n itself, for the gradient's adjoint steps
                    float *lo = lapout + shot_off + mp;
                    if (vec && gx + 3 < geo.nx) {
                        *reinterpret_cast<float4 *>(lo) = make_float4(acc[0][i][0], acc[0][i][1], acc[0][i][2], acc[0][i][3]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (gx + k < geo.nx) lo[k] = acc[0][i][k];
                    }
                }
                if (rec && z == geo.rec_z) {
                    float *rp = rec + ((int64_t)sh * geo.ny + y) * geo.nx + gx;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (gx + k < geo.nx) rp[k] = res[k];
                }
                if constexpr (ADJ) {
                    if (has_grad) {
                        const int64_t gi = ((int64_t)z * geo.ny + y) * geo.nx + gx;
                        if (gbulk) {
#pragma unroll
                            for (int k = 0; k < 4; ++k) gb[(ry0 + i) * TX + 4 * tx + k] = gd[k];
                        } else if (geo.gss == 0) {
                            // one slice for all shots: other CTAs add to the same points
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                if (gx + k < geo.nx) atomicAdd(adj.grad + gi + k, gd[k]);
                        } else {
                            // this shot's own slice: no other thread touches these points
                            double *gp = adj.grad + (int64_t)sh * geo.gss + gi;
                            if (adj.gvec && gx + 3 < geo.nx) {
                                double2 *g2 = reinterpret_cast<double2 *>(gp);
                                double2 a = g2[0], b = g2[1];
                                a.x += gd[0]; a.y += gd[1]; b.x += gd[2]; b.y += gd[3];
                                g2[0] = a;
                                g2[1] = b;
                            } else {
#pragma unroll
                                for (int k = 0; k < 4; ++k)
                                    if (gx + k < geo.nx) gp[k] += gd[k];
                            }
                        }
                    }
                }
            }
            if constexpr (ADJ) {
                if (gbulk) {
                    // the terms reach the async proxy, then each row's first
                    // thread adds the row's valid points (an even count: nx
                    // and x0 are even) with one bulk reduction
                    ptx::fence_proxy_async_smem();
                    __syncwarp();
                    if (tx == 0) {
#pragma unroll
                        for (int i = 0; i < PY; ++i) {
                            const int y = y0 + ry0 + i;
                            if (y < geo.ny && x0 < geo.nx) {
                                const int n = min(TX, geo.nx - x0);
                                bulk_add_f64(adj.grad + ((int64_t)z * geo.ny + y) * geo.nx + x0, gb + (ry0 + i) * TX,
                                             (uint32_t)n * 8u);
                            }
                        }
                        bulk_commit();
                    }
                }
            }
        }
#pragma unroll
        for (int kk = 0; kk < W - 1; ++kk)
#pragma unroll
            for (int i = 0; i < PY; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[kk][i][k] = acc[kk + 1][i][k];
#pragma unroll
        for (int i = 0; i < PY; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[W - 1][i][k] = 0.f;
    }
    // this thread's reductions are complete before the CTA exits
    if constexpr (ADJ)
        if (gbulk && tx == 0) bulk_wait_all();
}

// Adjoint step.  Ring stage s holds the planes lam^{n+1}, m, a^n (with halo)
// of input plane j and the interior tiles lam^{n+2} and lam^{n+1} of the
// output plane zo = j - 2R that plane j completes.
template <int R, int TX, int TY, int S>
struct AdjGeom {
    using G = Geom<R, TX, TY, 1, S>;
    using I = Interior<R, TX>;
    static constexpr int PL = (G::PLANE + 31) & ~31;   // padded plane stride
    static constexpr int MT = (I::BXI * TY + 31) & ~31;
    static constexpr int OFF_L2 = 3 * PL, OFF_L1 = OFF_L2 + MT;
    static constexpr int STAGE = OFF_L1 + MT;
    // [ring | q plane | sponge tables | barriers | abort flag]
    static constexpr size_t OFF_Q = (size_t)S * STAGE;
    static constexpr size_t OFF_GX = OFF_Q + PL;
    static constexpr size_t OFF_GY = OFF_GX + ((G::BX + 3) & ~3);
    static constexpr size_t OFF_BAR = OFF_GY + ((G::BY + 3) & ~3);
    static constexpr size_t SMEM = 128 + OFF_BAR * 4 + S * 8 + 16;
};

// LAPIN: the gradient term reads L a^n as a completed tile (written by the
// forward step that produced a^{n+1}) instead of staging a^n and applying
// the stencil here; the a^n plane's ring slot then holds that tile.
template <int R, int TX, int TY, int S, bool LAPIN>
__global__ void __launch_bounds__(Geom<R, TX, TY, 1, S>::NT, 2)
    wave_adj_kernel(const __grid_constant__ CUtensorMap tlam, const __grid_constant__ CUtensorMap tm,
                    const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tl2,
                    const __grid_constant__ CUtensorMap tl1, const __grid_constant__ StarCoef cf,
                    const __grid_constant__ WaveGeo geo, float *__restrict__ lprev,
                    const float *__restrict__ resid, double *__restrict__ grad, int has_a, int tz,
                    int nzc, int gvec, unsigned *err)
{
    constexpr int PY = 1;
    using G = Geom<R, TX, TY, PY, S>;
    using A = AdjGeom<R, TX, TY, S>;
    using I = Interior<R, TX>;
    constexpr int W = G::W;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *base = reinterpret_cast<float *>(smem_align128(smem_raw));
    float *qbuf = base + A::OFF_Q;
    float *gxt = base + A::OFF_GX;
    float *gyt = base + A::OFF_GY;
    uint64_t *full = reinterpret_cast<uint64_t *>(base + A::OFF_BAR);
    int &abort_flag = *reinterpret_cast<int *>(full + S);

    const int tid = threadIdx.x;
    const int tx = tid % G::NTX, ty = tid / G::NTX;
    const int sh = blockIdx.z / nzc, zc = blockIdx.z % nzc;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, zb = zc * tz;
    const int nzt = min(tz, geo.nz - zb);
    const int P = nzt + 2 * R;
    const int ry0 = ty * PY;
    const int gx = x0 + 4 * tx;
    const uint32_t plane_bytes = (has_a && !LAPIN ? 3u : 2u) * G::PLANE * sizeof(float);

    for (int c = tid; c < G::BX; c += G::NT) gxt[c] = sponge(x0 + c - R, geo.nx, geo.sponge_w, geo.sponge_a);
    for (int rr = tid; rr < G::BY; rr += G::NT) gyt[rr] = sponge(y0 + rr - R, geo.ny, geo.sponge_w, geo.sponge_a);
    if (tid == 0) {
        ptx::prefetch_tmap(&tlam);
        ptx::prefetch_tmap(&tm);
        ptx::prefetch_tmap(&tl2);
        ptx::prefetch_tmap(&tl1);
        if (has_a) ptx::prefetch_tmap(&ta);  // a^n planes, or L a^n tiles
#pragma unroll
        for (int s = 0; s < S; ++s) ptx::mbar_init(&full[s], 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();
    auto issue = [&](int j, int s) {
        float *st = base + (size_t)s * A::STAGE;
        const bool inner = j >= 2 * R;
        const uint32_t tiles = inner ? (LAPIN && has_a ? 3u : 2u) : 0u;
        ptx::mbar_arrive_expect_tx(&full[s], plane_bytes + tiles * I::BXI * TY * 4u);
        ptx::tma_load_4d(st, &tlam, x0, y0, zb + j, sh, &full[s]);
        ptx::tma_load_3d(st + A::PL, &tm, x0, y0, zb + j, &full[s]);
        if (has_a && !LAPIN) ptx::tma_load_4d(st + 2 * A::PL, &ta, x0, y0, zb + j, sh, &full[s]);
        if (inner) {
            const int zp = zb + j - R;
            const int xs = x0 + (R & ~3);
            ptx::tma_load_4d(st + A::OFF_L2, &tl2, xs, y0 + R, zp, sh, &full[s]);
            ptx::tma_load_4d(st + A::OFF_L1, &tl1, xs, y0 + R, zp, sh, &full[s]);
            if (LAPIN && has_a) ptx::tma_load_4d(st + 2 * A::PL, &ta, xs, y0 + R, zp, sh, &full[s]);
        }
    };
    if (tid == 0)
        for (int j = 0; j < S && j < P; ++j) issue(j, j);

    float accq[W][PY][4], acca[W][PY][4];
#pragma unroll
    for (int kk = 0; kk < W; ++kk)
#pragma unroll
        for (int k = 0; k < 4; ++k) accq[kk][0][k] = acca[kk][0][k] = 0.f;
    float gxs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) gxs[k] = gxt[4 * tx + R + k];
    const float gys0 = gyt[ry0 + R];
    const int64_t shot_off = (int64_t)sh * geo.ss;

    // Input plane j; the oldest partial sums (output plane j - 2R) are in
    // queue slot 0.  Returns false when the CTA aborts.  (Rotating the two
    // queues instead of shifting them, as the sweeps do, spills registers
    // here and was measured slower.)
    auto plane = [&](int j) -> bool {
        constexpr int Q = 0;
        const int s = j % S;
        const float *st = base + (size_t)s * A::STAGE;
        const int zo = j - 2 * R;
        const bool ok = ptx::mbar_wait_bounded(&full[s], (uint32_t)(j / S) & 1u, err);
        if (ok) {
            // q = m * g * lam^{n+1} over the whole staged plane, four columns
            // per item (the staged rows are 16-byte multiples)
            const float gzp = sponge(zb + j - R, geo.nz, geo.sponge_w, geo.sponge_a);
            constexpr int BX4 = G::BX / 4;
            for (int e4 = tid; e4 < BX4 * G::BY; e4 += G::NT) {
                const int c4 = e4 % BX4, rr = e4 / BX4;
                const int e = rr * G::BX + 4 * c4;
                const float4 lv = *reinterpret_cast<const float4 *>(st + e);
                const float4 mv = *reinterpret_cast<const float4 *>(st + A::PL + e);
                const float4 gx = *reinterpret_cast<const float4 *>(gxt + 4 * c4);
                const float gy = gyt[rr];
                float4 q;
                q.x = mv.x * (gx.x * gy * gzp) * lv.x;
                q.y = mv.y * (gx.y * gy * gzp) * lv.y;
                q.z = mv.z * (gx.z * gy * gzp) * lv.z;
                q.w = mv.w * (gx.w * gy * gzp) * lv.w;
                *reinterpret_cast<float4 *>(qbuf + e) = q;
            }
        } else {
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) return false;
        float l2v[4], l1v[4], lav[4];
        {
            float unused[PY][4];
            star_plane<R, PY, G::BX, G::NV, Q>(qbuf, cf, accq, unused, tx, ry0);
            if (!LAPIN && has_a) star_plane<R, PY, G::BX, G::NV, Q>(st + 2 * A::PL, cf, acca, unused, tx, ry0);
            if (zo >= 0) {
                load_center<I::OFF>(st + A::OFF_L2 + ry0 * I::BXI + 4 * tx, l2v);
                load_center<I::OFF>(st + A::OFF_L1 + ry0 * I::BXI + 4 * tx, l1v);
                if (LAPIN && has_a) load_center<I::OFF>(st + 2 * A::PL + ry0 * I::BXI + 4 * tx, lav);
            }
        }
        __syncthreads();
        if (tid == 0 && j + S < P) issue(j + S, s);
        if (zo >= 0) {
            const int z = zb + zo;
            const int y = y0 + ry0;
            if (y < geo.ny && gx < geo.nx) {
                const float gzv = sponge(z, geo.nz, geo.sponge_w, geo.sponge_a);
                const int64_t mp = (int64_t)(z + R) * geo.pz + (int64_t)(y + R) * geo.py + (gx + R);
                float *lp = lprev + shot_off + mp;
                const int64_t gi = ((int64_t)z * geo.ny + y) * geo.nx + gx;
                const bool at_rec = resid && z == geo.rec_z;
                double gd[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (gx + k >= geo.nx) break;
                    const float g = gxs[k] * gys0 * gzv;
                    float v = 2.f * g * l1v[k] + accq[Q][0][k] - g * g * l2v[k];
                    if (at_rec) v += resid[((int64_t)sh * geo.ny + y) * geo.nx + gx + k];
                    lp[k] = v;
                    // the step's term in FP32 (its operands are FP32), accumulated in FP64
                    if (has_a) gd[k] = widen(g * l1v[k] * (LAPIN ? lav[k] : acca[Q][0][k]));
                }
                if (has_a) {
                    if (geo.gss == 0) {
                        // one slice for all shots: other CTAs add to the same points
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (gx + k < geo.nx) atomicAdd(grad + gi + k, gd[k]);
                    } else {
                        // this shot's own slice: no other thread touches these points
                        double *gp = grad + (int64_t)sh * geo.gss + gi;
                        if (gvec && gx + 3 < geo.nx) {
                            double2 *g2 = reinterpret_cast<double2 *>(gp);
                            double2 a = g2[0], b = g2[1];
                            a.x += gd[0]; a.y += gd[1]; b.x += gd[2]; b.y += gd[3];
                            g2[0] = a;
                            g2[1] = b;
                        } else {
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                if (gx + k < geo.nx) gp[k] += gd[k];
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int kk = 0; kk < W - 1; ++kk)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                accq[kk][0][k] = accq[kk + 1][0][k];
                acca[kk][0][k] = acca[kk + 1][0][k];
            }
#pragma unroll
        for (int k = 0; k < 4; ++k) accq[W - 1][0][k] = acca[W - 1][0][k] = 0.f;
        return true;
    };
    for (int j = 0; j < P; ++j)
        if (!plane(j)) return;
}

__global__ void model_kernel(WaveGeo geo, const float *__restrict__ v, float *__restrict__ m, float s)
{
    const int r = geo.r;
    const int64_t X = geo.nx + 2 * r, Y = geo.ny + 2 * r, Z = geo.nz + 2 * r;
    const int64_t total = X * Y * Z;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t xx = i % X, yy = (i / X) % Y, zz = i / (X * Y);
        const int64_t x = xx - r, y = yy - r, z = zz - r;
        float val = 0.f;
        if (x >= 0 && x < geo.nx && y >= 0 && y < geo.ny && z >= 0 && z < geo.nz) {
            const float vv = v[(z * geo.ny + y) * geo.nx + x];
            val = vv * vv * s;
        }
        m[zz * geo.pz + yy * geo.py + xx] = val;
    }
}

// grad[z][y][x] /= m at the interior point (FP64): the scaled adjoint's sum
// of mu^{n+1} (L a^n) turned into dJ/dm.
__global__ void divide_m_kernel(WaveGeo geo, const float *__restrict__ m, double *__restrict__ grad)
{
    const int r = geo.r;
    const int64_t n = (int64_t)geo.nx * geo.ny * geo.nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % geo.nx, y = (i / geo.nx) % geo.ny, z = i / ((int64_t)geo.nx * geo.ny);
        grad[i] = grad[i] / (double)m[(z + r) * geo.pz + (y + r) * geo.py + x + r];
    }
}

__global__ void chain_kernel(const double *__restrict__ gm, const float *__restrict__ v,
                             double *__restrict__ gv, int64_t n, double s)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        gv[i] = gm[i] * 2.0 * (double)v[i] * s;
}

__global__ void sum_kernel(const double *__restrict__ slices, int nslices, int64_t stride, int64_t n,
                           double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = slices[i];
        for (int s = 1; s < nslices; ++s) acc += slices[(int64_t)s * stride + i];
        out[i] = acc;
    }
}

__global__ void dot_kernel(const float *__restrict__ a, const float *__restrict__ b, int64_t n,
                           double *__restrict__ res)
{
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < blockDim.x / 32 ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(res, acc);
    }
}

constexpr int kFwdTX = 64, kFwdTY = 16, kFwdPY = 1, kFwdS = 3, kFwdTZ = 128;
constexpr int kAdjTX = 64, kAdjTY = 16, kAdjS = 2, kAdjTZ = 128;

template <int R>
cudaError_t fwd_r(const WaveGeo &g, const StarCoef &cf, const float *m, const float *p_cur,
                  const float *p_prev, float *p_next, const float *amp, float *rec, float *lapout,
                  cudaStream_t st, const float *lap_in = nullptr, const AdjArgs *adj = nullptr)
{
    using G = Geom<R, kFwdTX, kFwdTY, kFwdPY, kFwdS>;
    using I = Interior<R, kFwdTX>;
    const int X = g.nx + 2 * R, Y = g.ny + 2 * R, Z = g.nz + 2 * R;
    CUtensorMap mcur, mm, mprev, mctr, mlap;
    if (!encode_tmap_4d(&mcur, p_cur, X, Y, Z, g.nshots, g.py, g.pz, g.ss, G::BX, G::BY, 1) ||
        !encode_tmap_3d(&mm, m, X, Y, Z, g.py, g.pz, I::BXI, kFwdTY, 1) ||
        !encode_tmap_4d(&mprev, p_prev, X, Y, Z, g.nshots, g.py, g.pz, g.ss, I::BXI, kFwdTY, 1) ||
        !encode_tmap_4d(&mctr, p_cur, X, Y, Z, g.nshots, g.py, g.pz, g.ss, I::BXI, kFwdTY, 1))
        return cudaErrorInvalidValue;
    if (lap_in) {
        if (!encode_tmap_4d(&mlap, lap_in, X, Y, Z, g.nshots, g.py, g.pz, g.ss, I::BXI, kFwdTY, 1))
            return cudaErrorInvalidValue;
    } else {
        mlap = mctr;  // not read
    }
    const int mode = adj ? K_ADJ_SCALED : lapout ? K_FWD_LAP : K_FWD;
    auto kern = mode == K_ADJ_SCALED ? wave_fwd_kernel<R, kFwdTX, kFwdTY, kFwdPY, kFwdS, K_ADJ_SCALED>
                : mode == K_FWD_LAP  ? wave_fwd_kernel<R, kFwdTX, kFwdTY, kFwdPY, kFwdS, K_FWD_LAP>
                                     : wave_fwd_kernel<R, kFwdTX, kFwdTY, kFwdPY, kFwdS, K_FWD>;
    using FA = FwdGeom<R, kFwdTX, kFwdTY, kFwdPY, kFwdS, K_ADJ_SCALED>;
    // the adjoint's gradient buffers only where its bulk reductions run
    const bool gbulk = adj && adj->grad && g.gss == 0 && adj->gbulk;
    const size_t smem = mode == K_ADJ_SCALED ? FA::SMEM - (gbulk ? 0 : FA::GB_BYTES)
                        : mode == K_FWD_LAP  ? FwdGeom<R, kFwdTX, kFwdTY, kFwdPY, kFwdS, K_FWD_LAP>::SMEM
                                             : FwdGeom<R, kFwdTX, kFwdTY, kFwdPY, kFwdS, K_FWD>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // z chunks of kFwdTZ planes.  The adjoint step on a grid whose CTAs fill
    // at most one wave splits z finer, into about three waves, so that the
    // SMs left with one CTA do not idle while the others finish two (2 x
    // 256^3: 219 -> 207 us per step; the forward forms gained nothing).
    const int cols = (g.nx + kFwdTX - 1) / kFwdTX * ((g.ny + kFwdTY - 1) / kFwdTY) * g.nshots;
    int tz = kFwdTZ;
    if (mode == K_ADJ_SCALED) {
        // resident CTAs of this launch on the current device (cached per
        // device, without / with the gradient buffers)
        constexpr int kDevs = 16;
        static int slots[kDevs][2] = {};
        int dev = 0, sl_local = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
        int &sl = dev >= 0 && dev < kDevs ? slots[dev][gbulk ? 1 : 0] : sl_local;
        if (sl == 0) {
            int sms = 0, per_sm = 0;
            if (dev >= 0 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::NT, smem) == cudaSuccess)
                sl = sms * per_sm > 0 ? sms * per_sm : -1;
            else
                sl = -1;
        }
        if (sl > 0 && cols * ((g.nz + tz - 1) / tz) <= sl) {
            const int k = (3 * sl + cols / 2) / cols;  // chunks per column for about three waves
            tz = k > 0 ? (g.nz + k - 1) / k : tz;
            if (tz < 2 * R) tz = 2 * R;
        }
    }
    const int nzc = (g.nz + tz - 1) / tz;
    const dim3 grid((g.nx + kFwdTX - 1) / kFwdTX, (g.ny + kFwdTY - 1) / kFwdTY, nzc * g.nshots);
    const int vec = (R % 4 == 0) && g.py % 4 == 0 && g.pz % 4 == 0 && g.ss % 4 == 0 &&
                    reinterpret_cast<uintptr_t>(p_next) % 16 == 0 && reinterpret_cast<uintptr_t>(lapout) % 16 == 0;
    const AdjArgs aa = adj ? *adj : AdjArgs{nullptr, nullptr, 0, 0};
    return launch_overlapped(kern, grid, dim3(G::NT), smem, st, mcur, mm, mprev, mctr, mlap, cf, g, p_next, amp, rec,
                             lapout, aa, tz, nzc, vec, device_error_word());
}

template <int R, bool LAPIN>
cudaError_t adj_r(const WaveGeo &g, const StarCoef &cf, const float *m, const float *lam_cur,
                  float *lam_prev, const float *resid, const float *a_n, double *grad, cudaStream_t st)
{
    using G = Geom<R, kAdjTX, kAdjTY, 1, kAdjS>;
    using A = AdjGeom<R, kAdjTX, kAdjTY, kAdjS>;
    using I = Interior<R, kAdjTX>;
    CUtensorMap ml, mm, ma, m2, m1;
    const int X = g.nx + 2 * R, Y = g.ny + 2 * R, Z = g.nz + 2 * R;
    if (!encode_tmap_4d(&ml, lam_cur, X, Y, Z, g.nshots, g.py, g.pz, g.ss, G::BX, G::BY, 1) ||
        !encode_tmap_3d(&mm, m, X, Y, Z, g.py, g.pz, G::BX, G::BY, 1) ||
        !encode_tmap_4d(&m2, lam_prev, X, Y, Z, g.nshots, g.py, g.pz, g.ss, I::BXI, kAdjTY, 1) ||
        !encode_tmap_4d(&m1, lam_cur, X, Y, Z, g.nshots, g.py, g.pz, g.ss, I::BXI, kAdjTY, 1))
        return cudaErrorInvalidValue;
    if (a_n) {
        // a^n planes with halo, or (LAPIN) interior tiles of L a^n
        if (!encode_tmap_4d(&ma, a_n, X, Y, Z, g.nshots, g.py, g.pz, g.ss, LAPIN ? I::BXI : G::BX,
                            LAPIN ? kAdjTY : G::BY, 1))
            return cudaErrorInvalidValue;
    } else {
        ma = ml;
    }
    auto kern = wave_adj_kernel<R, kAdjTX, kAdjTY, kAdjS, LAPIN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)A::SMEM);
    if (e != cudaSuccess) return e;
    const int tz = kAdjTZ;
    const int nzc = (g.nz + tz - 1) / tz;
    const dim3 grid((g.nx + kAdjTX - 1) / kAdjTX, (g.ny + kAdjTY - 1) / kAdjTY, nzc * g.nshots);
    // 32-byte aligned rows of four doubles: two double2 per thread
    const int gvec = g.nx % 4 == 0 && g.gss % 4 == 0 && reinterpret_cast<uintptr_t>(grad) % 32 == 0;
    kern<<<grid, G::NT, A::SMEM, st>>>(ml, mm, ma, m2, m1, cf, g, lam_prev, resid, grad, a_n ? 1 : 0,
                                       tz, nzc, gvec, device_error_word());
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_wave_fwd(const WaveGeo &g, const float *coeffs, const float *m, const float *p_cur,
                            const float *p_prev, float *p_next, const float *src_amp, float *rec,
                            cudaStream_t st, float *lapout)
{
    StarCoef cf{};
    for (int i = 0; i < 3 * (2 * g.r + 1); ++i) cf.c[i] = coeffs[i];
    switch (g.r) {
        case 1: return fwd_r<1>(g, cf, m, p_cur, p_prev, p_next, src_amp, rec, lapout, st);
        case 2: return fwd_r<2>(g, cf, m, p_cur, p_prev, p_next, src_amp, rec, lapout, st);
        case 3: return fwd_r<3>(g, cf, m, p_cur, p_prev, p_next, src_amp, rec, lapout, st);
        case 4: return fwd_r<4>(g, cf, m, p_cur, p_prev, p_next, src_amp, rec, lapout, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_wave_adj_scaled(const WaveGeo &g, const float *coeffs, const float *m, const float *mu_cur,
                                   float *mu_prev, const float *resid, const float *lap_a, double *grad,
                                   cudaStream_t st)
{
    StarCoef cf{};
    for (int i = 0; i < 3 * (2 * g.r + 1); ++i) cf.c[i] = coeffs[i];
    const AdjArgs adj{resid, lap_a ? grad : nullptr,
                      g.nx % 4 == 0 && g.gss % 4 == 0 && reinterpret_cast<uintptr_t>(grad) % 32 == 0,
                      g.nx % 2 == 0 && reinterpret_cast<uintptr_t>(grad) % 16 == 0};
    const float *lap = lap_a && grad ? lap_a : nullptr;
    switch (g.r) {
        case 1: return fwd_r<1>(g, cf, m, mu_cur, mu_prev, mu_prev, nullptr, nullptr, nullptr, st, lap, &adj);
        case 2: return fwd_r<2>(g, cf, m, mu_cur, mu_prev, mu_prev, nullptr, nullptr, nullptr, st, lap, &adj);
        case 3: return fwd_r<3>(g, cf, m, mu_cur, mu_prev, mu_prev, nullptr, nullptr, nullptr, st, lap, &adj);
        case 4: return fwd_r<4>(g, cf, m, mu_cur, mu_prev, mu_prev, nullptr, nullptr, nullptr, st, lap, &adj);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_wave_adj(const WaveGeo &g, const float *coeffs, const float *m, const float *lam_cur,
                            float *lam_prev, const float *resid, const float *a_n, double *grad,
                            cudaStream_t st, bool lapin)
{
    StarCoef cf{};
    for (int i = 0; i < 3 * (2 * g.r + 1); ++i) cf.c[i] = coeffs[i];
#define MMS_ADJ(R_)                                                                              \
    return lapin ? adj_r<R_, true>(g, cf, m, lam_cur, lam_prev, resid, a_n, grad, st)            \
                 : adj_r<R_, false>(g, cf, m, lam_cur, lam_prev, resid, a_n, grad, st);
    switch (g.r) {
        case 1: MMS_ADJ(1)
        case 2: MMS_ADJ(2)
        case 3: MMS_ADJ(3)
        case 4: MMS_ADJ(4)
        default: return cudaErrorInvalidValue;
    }
#undef MMS_ADJ
}

cudaError_t launch_model_from_velocity(const WaveGeo &g, const float *v, float *m, float dt, float h,
                                       cudaStream_t st)
{
    const float s = (dt * dt) / (h * h);
    model_kernel<<<152 * 8, 256, 0, st>>>(g, v, m, s);
    return cudaGetLastError();
}

cudaError_t launch_grad_to_velocity(const double *gm, const float *v, double *gv, int64_t n, float dt,
                                    float h, cudaStream_t st)
{
    const double s = ((double)dt * dt) / ((double)h * h);
    chain_kernel<<<152 * 8, 256, 0, st>>>(gm, v, gv, n, s);
    return cudaGetLastError();
}

cudaError_t launch_grad_divide_m(const WaveGeo &g, const float *m, double *grad, cudaStream_t st)
{
    divide_m_kernel<<<152 * 8, 256, 0, st>>>(g, m, grad);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(unsigned long long limit_ns, cudaStream_t st)
{
    wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns, device_error_word());
    return cudaGetLastError();
}

cudaError_t launch_sum_f64(const double *slices, int nslices, int64_t stride, int64_t n, double *out,
                           cudaStream_t st)
{
    sum_kernel<<<152 * 8, 256, 0, st>>>(slices, nslices, stride, n, out);
    return cudaGetLastError();
}

cudaError_t launch_dot_f64(const float *a, const float *b, int64_t n, double *res, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(res, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    dot_kernel<<<152 * 4, 256, 0, st>>>(a, b, n, res);
    return cudaGetLastError();
}

}  // namespace mms
