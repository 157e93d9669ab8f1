// abi.cu -- the C ABI of include/mms.h: argument validation, path and
// variant choice, TMA descriptor encoding, error reporting.
#include <cudaTypedefs.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>

#include "common.cuh"
#include "validate.cuh"
#include "wave.cuh"

namespace mms {

static thread_local std::string g_last_error;

mms_status fail(mms_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

mms_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(MMS_E_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// ---------------------------------------------------------- tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool encode_tmap_3d(CUtensorMap *map, const float *base, int64_t X, int64_t Y, int64_t Z,
                    int64_t py, int64_t pz, int bx, int by, int bz, bool swizzle128)
{
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)Z};
    cuuint64_t strides[2] = {(cuuint64_t)py * 4, (cuuint64_t)pz * 4};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_tmap_4d(CUtensorMap *map, const float *base, int64_t X, int64_t Y, int64_t Z,
                    int64_t W, int64_t py, int64_t pz, int64_t pw, int bx, int by, int bz)
{
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[4] = {(cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)Z, (cuuint64_t)W};
    cuuint64_t strides[3] = {(cuuint64_t)py * 4, (cuuint64_t)pz * 4, (cuuint64_t)pw * 4};
    cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ------------------------------------------------------- variant table
// Registered variants (mms_set_variant): kUnset = none registered (the
// built-in table below decides), kCleared = explicitly none, else the variant.
constexpr int kUnset = -1, kCleared = -2;
static std::mutex g_var_mu;
static int g_tuned[4][kMaxR + 1][8];
static bool g_tuned_init = false;

// Built-in table: the autotuner's committed rows (tuned.json), compiled in
// by build.py; a row applies on a device whose name is the row's GPU name.
struct TunedRow {
    const char *gpu;
    int shape, r, path, variant;
};
#include "tuned_defaults.inc"

constexpr int kMaxDevices = 64;
static int g_dev_row_gpu[kMaxDevices];  // per device: 0 = unknown, 1 = no rows, 2 + i = rows of GPU name i
static bool g_dev_init = false;

// Index (into kTunedRows) of the first row whose GPU name is the current
// device's, or -1 (no device, or no rows for it).  Looked up once per device.
static int device_rows()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return -1;
    }
    {
        std::lock_guard<std::mutex> lk(g_var_mu);
        if (!g_dev_init) {
            for (int &x : g_dev_row_gpu) x = 0;
            g_dev_init = true;
        }
        if (g_dev_row_gpu[dev] != 0) return g_dev_row_gpu[dev] - 2;
    }
    int found = -1;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) {
        for (size_t i = 0; i < sizeof(kTunedRows) / sizeof(kTunedRows[0]); ++i)
            if (kTunedRows[i].shape >= 0 && strcmp(kTunedRows[i].gpu, p.name) == 0) {
                found = (int)i;
                break;
            }
    } else {
        cudaGetLastError();
    }
    std::lock_guard<std::mutex> lk(g_var_mu);
    g_dev_row_gpu[dev] = found + 2;
    return found;
}

static int builtin_variant(int shape, int r, int path)
{
    const int first = device_rows();
    if (first < 0) return -1;
    const char *gpu = kTunedRows[first].gpu;
    for (size_t i = first; i < sizeof(kTunedRows) / sizeof(kTunedRows[0]); ++i) {
        const TunedRow &t = kTunedRows[i];
        if (strcmp(t.gpu, gpu) == 0 && t.shape == shape && t.r == r && t.path == path) return t.variant;
    }
    return -1;
}

// The tuned variant of (shape, r, path): the registered one, else the
// built-in row for this device, else -1.
static int tuned_variant(int shape, int r, int path)
{
    int reg;
    {
        std::lock_guard<std::mutex> lk(g_var_mu);
        if (!g_tuned_init) {
            for (auto &a : g_tuned)
                for (auto &b : a)
                    for (int &c : b) c = kUnset;
            g_tuned_init = true;
        }
        reg = g_tuned[shape][r][path];
    }
    if (reg >= 0) return reg;
    if (reg == kCleared) return -1;
    return builtin_variant(shape, r, path);
}

static int num_variants(int shape, int r, int path)
{
    if (shape < 0 || shape > 3 || r < 1 || r > kMaxR) return 0;
    switch (path) {
        case MMS_PATH_CUDA_CORE:
            return shape == MMS_STAR ? star_cc_variants() : shape == MMS_BOX ? box_cc_variants() : plane_cc_variants();
        case MMS_PATH_NAIVE: return 1;
        case MMS_PATH_TF32:
        case MMS_PATH_3XTF32:
        case MMS_PATH_BF16X3: return band_tc_supported(shape, r, path) ? band_tc_variants(shape, r, path) : 0;
        default: return 0;
    }
}

// The registered (tuned) variant, else variant 0.
static int default_variant(int shape, int r, int path)
{
    const int t = tuned_variant(shape, r, path);
    return t >= 0 && t < num_variants(shape, r, path) ? t : 0;
}

static bool tma_ok(const float *in, int64_t ipy, int64_t ipz)
{
    return (reinterpret_cast<uintptr_t>(in) % 16) == 0 && (ipy % 4) == 0 && (ipz % 4) == 0;
}

// AUTO: the tensor-core BF16x3 path where a tuned variant for it exists
// (the autotuner records one only where it beats the CUDA-core path; the
// built-in table carries them for the GPUs it was tuned on), else the TMA
// CUDA-core path, else the naive path for unaligned pitches.
static int auto_path(int shape, int r, bool aligned)
{
    if (!aligned) return MMS_PATH_NAIVE;
    if (band_tc_supported(shape, r, MMS_PATH_BF16X3) && tuned_variant(shape, r, MMS_PATH_BF16X3) >= 0)
        return MMS_PATH_BF16X3;
    return MMS_PATH_CUDA_CORE;
}

static bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + nb && b0 < a0 + na;
}

static mms_status apply(const mms_stencil_desc *d, const float *in, float *out, void *stream)
{
    if (!d) return fail(MMS_E_ARG, "null descriptor");
    const int shape = d->shape, r = d->radius;
    if (shape < MMS_STAR || shape > MMS_BOX2D) return fail(MMS_E_ARG, "shape %d is not STAR, BOX, STAR2D or BOX2D", shape);
    if (r < 1 || r > kMaxR) return fail(MMS_E_ARG, "radius %d outside 1..%d", r, kMaxR);
    if (!d->coeffs) return fail(MMS_E_ARG, "null coefficient array");
    if (d->nx < 0 || d->ny < 0 || d->nz < 0) return fail(MMS_E_ARG, "negative size");
    if (d->nx >= (1ll << 30) || d->ny >= (1ll << 30) || d->nz >= (1ll << 30))
        return fail(MMS_E_ARG, "size above 2^30");
    if (d->path < MMS_PATH_AUTO || d->path > MMS_PATH_NAIVE) return fail(MMS_E_ARG, "unknown path %d", d->path);
    if (d->nx == 0 || d->ny == 0 || d->nz == 0) return MMS_OK;
    if (!in || !out) return fail(MMS_E_ARG, "null grid pointer");
    // planar shapes: nz independent planes, padded in x and y only
    const int64_t X = d->nx + 2 * r, Y = d->ny + 2 * r, Z = d->nz + (is_planar(shape) ? 0 : 2 * r);
    int64_t ipy, ipz, opy, opz;
    if (!resolve_pitches(X, Y, Z, d->in_pitch_y, d->in_pitch_z, &ipy, &ipz) ||
        !resolve_pitches(d->nx, d->ny, d->nz, d->out_pitch_y, d->out_pitch_z, &opy, &opz))
        return fail(MMS_E_ARG, "pitches not positive or spanning more than 2^46 elements");
    if (ipy < X || ipz < Y * ipy) return fail(MMS_E_ARG, "input pitches (%lld, %lld) below the padded extents", (long long)ipy, (long long)ipz);
    if (opy < d->nx || opz < d->ny * opy) return fail(MMS_E_ARG, "output pitches (%lld, %lld) below the interior extents", (long long)opy, (long long)opz);
    const size_t in_bytes = (size_t)((Z - 1) * ipz + (Y - 1) * ipy + X) * 4;
    const size_t out_bytes = (size_t)((d->nz - 1) * opz + (d->ny - 1) * opy + d->nx) * 4;
    if (overlaps(in, in_bytes, out, out_bytes)) return fail(MMS_E_ARG, "input and output overlap");
    if (d->variant < -1) return fail(MMS_E_ARG, "variant %d", d->variant);

    Sweep s{shape, r, d->nx, d->ny, d->nz, in, ipy, ipz, out, opy, opz, d->coeffs, d->variant,
            reinterpret_cast<cudaStream_t>(stream)};
    int path = d->path;
    const bool aligned = tma_ok(in, ipy, ipz);
    if (path == MMS_PATH_AUTO) path = auto_path(shape, r, aligned);
    if (path == MMS_PATH_NAIVE) {
        cudaError_t e = launch_naive(s);
        return e == cudaSuccess ? MMS_OK : cuda_fail(e, "naive sweep launch");
    }
    if (!aligned)
        return fail(MMS_E_ALIGN, "TMA path needs a 16-byte aligned input and pitches that are multiples of 4 floats");
    const int nvar = num_variants(shape, r, path);
    if (nvar == 0) return fail(MMS_E_UNSUPPORTED, "path %d does not support shape %d radius %d", path, shape, r);
    int v = d->variant >= 0 ? d->variant : default_variant(shape, r, path);
    if (v >= nvar) return fail(MMS_E_ARG, "variant %d of %d", v, nvar);
    CUtensorMap map;
    if (path == MMS_PATH_CUDA_CORE) {
        int bx, by;
        if (shape == MMS_STAR) star_cc_box(r, v, &bx, &by);
        else if (shape == MMS_BOX) box_cc_box(r, v, &bx, &by);
        else plane_cc_box(r, v, &bx, &by);
        if (!encode_tmap_3d(&map, in, X, Y, Z, ipy, ipz, bx, by, 1))
            return fail(MMS_E_CUDA, "cuTensorMapEncodeTiled refused the input grid");
        cudaError_t e = shape == MMS_STAR ? launch_star_cc(s, map, v)
                        : shape == MMS_BOX ? launch_box_cc(s, map, v)
                                           : launch_plane_cc(s, map, v);
        return e == cudaSuccess ? MMS_OK : cuda_fail(e, "CUDA-core sweep launch");
    }
    int bx, by, bz, swz;
    band_tc_box(shape, r, path, v, &bx, &by, &bz, &swz);
    if (!encode_tmap_3d(&map, in, X, Y, Z, ipy, ipz, bx, by, bz, swz != 0))
        return fail(MMS_E_CUDA, "cuTensorMapEncodeTiled refused the input grid");
    // The two-pass star's x/y partial sums go through a temporary grid
    // (stream-ordered allocation from the device's default memory pool).
    float *scratch = nullptr;
    s.variant = v;
    const size_t sb = band_tc_scratch_bytes(s);
    if (sb) {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), sb, s.stream);
        if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
    }
    cudaError_t e = launch_band_tc(s, path, map, v, scratch);
    if (scratch) {
        cudaError_t f = cudaFreeAsync(scratch, s.stream);
        if (e == cudaSuccess) e = f;
    }
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "tensor-core sweep launch");
}

cudaError_t launch_f64(int shape, int r, const double *coeffs, int ncoef, const double *in, int64_t ipy, int64_t ipz,
                       double *out, int64_t opy, int64_t opz, int64_t nx, int64_t ny, int64_t nz, cudaStream_t st);

static int n_coeffs(int shape, int r)
{
    const int w = 2 * r + 1;
    switch (shape) {
        case MMS_STAR: return 3 * w;
        case MMS_BOX: return w * w * w;
        case MMS_STAR2D: return 2 * w;
        default: return w * w;
    }
}

static mms_status apply_f64(const mms_stencil_desc *d, const double *coeffs, const double *in, double *out,
                            void *stream)
{
    if (!d) return fail(MMS_E_ARG, "null descriptor");
    const int shape = d->shape, r = d->radius;
    if (shape < MMS_STAR || shape > MMS_BOX2D) return fail(MMS_E_ARG, "shape %d is not STAR, BOX, STAR2D or BOX2D", shape);
    if (r < 1 || r > kMaxR) return fail(MMS_E_ARG, "radius %d outside 1..%d", r, kMaxR);
    if (!coeffs) return fail(MMS_E_ARG, "null coefficient array");
    if (d->nx < 0 || d->ny < 0 || d->nz < 0) return fail(MMS_E_ARG, "negative size");
    if (d->nx >= (1ll << 30) || d->ny >= (1ll << 30) || d->nz >= (1ll << 30))
        return fail(MMS_E_ARG, "size above 2^30");
    if (d->path != MMS_PATH_AUTO && d->path != MMS_PATH_CUDA_CORE)
        return fail(MMS_E_UNSUPPORTED, "FP64 sweeps run on the CUDA cores only (path %d)", d->path);
    if (d->nx == 0 || d->ny == 0 || d->nz == 0) return MMS_OK;
    if (!in || !out) return fail(MMS_E_ARG, "null grid pointer");
    if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % 8)
        return fail(MMS_E_ALIGN, "FP64 grids must be 8-byte aligned");
    const int64_t X = d->nx + 2 * r, Y = d->ny + 2 * r, Z = d->nz + (is_planar(shape) ? 0 : 2 * r);
    int64_t ipy, ipz, opy, opz;
    if (!resolve_pitches(X, Y, Z, d->in_pitch_y, d->in_pitch_z, &ipy, &ipz) ||
        !resolve_pitches(d->nx, d->ny, d->nz, d->out_pitch_y, d->out_pitch_z, &opy, &opz))
        return fail(MMS_E_ARG, "pitches not positive or spanning more than 2^46 elements");
    if (ipy < X || ipz < Y * ipy) return fail(MMS_E_ARG, "input pitches (%lld, %lld) below the padded extents", (long long)ipy, (long long)ipz);
    if (opy < d->nx || opz < d->ny * opy) return fail(MMS_E_ARG, "output pitches (%lld, %lld) below the interior extents", (long long)opy, (long long)opz);
    const size_t in_bytes = (size_t)((Z - 1) * ipz + (Y - 1) * ipy + X) * 8;
    const size_t out_bytes = (size_t)((d->nz - 1) * opz + (d->ny - 1) * opy + d->nx) * 8;
    if (overlaps(in, in_bytes, out, out_bytes)) return fail(MMS_E_ARG, "input and output overlap");
    cudaError_t e = launch_f64(shape, r, coeffs, n_coeffs(shape, r), in, ipy, ipz, out, opy, opz, d->nx, d->ny, d->nz,
                               reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "FP64 sweep launch");
}

// The sweep of apply() on grids in host memory: z-slabs of the input (with
// their 2r halo planes) are copied in, swept and copied back, pipelined over
// two device slab buffers and three streams -- copy in and copy out on
// streams of the call's own, the sweeps on the caller's stream, which at
// return waits for the last copy back.
static mms_status apply_host(const mms_stencil_desc *d, const float *in, float *out, void *stream)
{
    if (!d) return fail(MMS_E_ARG, "null descriptor");
    const int r = d->radius;
    if (d->shape < MMS_STAR || d->shape > MMS_BOX2D)
        return fail(MMS_E_ARG, "shape %d is not STAR, BOX, STAR2D or BOX2D", d->shape);
    const int rz = is_planar(d->shape) ? 0 : r;  // z halo of the input
    if (r < 1 || r > kMaxR) return fail(MMS_E_ARG, "radius %d outside 1..%d", r, kMaxR);
    if (!d->coeffs) return fail(MMS_E_ARG, "null coefficient array");
    if (d->nx < 0 || d->ny < 0 || d->nz < 0) return fail(MMS_E_ARG, "negative size");
    if (d->nx >= (1ll << 30) || d->ny >= (1ll << 30) || d->nz >= (1ll << 30))
        return fail(MMS_E_ARG, "size above 2^30");
    if (d->path < MMS_PATH_AUTO || d->path > MMS_PATH_NAIVE) return fail(MMS_E_ARG, "unknown path %d", d->path);
    if (d->variant < -1) return fail(MMS_E_ARG, "variant %d", d->variant);
    if (d->nx == 0 || d->ny == 0 || d->nz == 0) return MMS_OK;
    if (!in || !out) return fail(MMS_E_ARG, "null grid pointer");
    const int64_t X = d->nx + 2 * r, Y = d->ny + 2 * r, Z = d->nz + 2 * rz;
    int64_t ipy, ipz, opy, opz;
    if (!resolve_pitches(X, Y, Z, d->in_pitch_y, d->in_pitch_z, &ipy, &ipz) ||
        !resolve_pitches(d->nx, d->ny, d->nz, d->out_pitch_y, d->out_pitch_z, &opy, &opz))
        return fail(MMS_E_ARG, "pitches not positive or spanning more than 2^46 elements");
    if (ipy < X || ipz < Y * ipy) return fail(MMS_E_ARG, "input pitches below the padded extents");
    if (opy < d->nx || opz < d->ny * opy) return fail(MMS_E_ARG, "output pitches below the interior extents");
    if (ipy % 4 || ipz % 4) return fail(MMS_E_ALIGN, "host input pitches must be multiples of 4 floats");
    const size_t in_bytes = (size_t)((Z - 1) * ipz + (Y - 1) * ipy + X) * 4;
    const size_t out_bytes = (size_t)((d->nz - 1) * opz + (d->ny - 1) * opy + d->nx) * 4;
    if (overlaps(in, in_bytes, out, out_bytes)) return fail(MMS_E_ARG, "input and output overlap");

    // slab depth: about eight slabs, 8..128 planes
    int64_t tz = ((d->nz + 7) / 8 + 7) / 8 * 8;
    tz = tz < 8 ? 8 : tz > 128 ? 128 : tz;
    if (tz > d->nz) tz = d->nz;
    const int64_t nslab = (d->nz + tz - 1) / tz;
    const size_t in_slab = (size_t)(tz + 2 * rz) * ipz * 4, out_slab = (size_t)tz * opz * 4;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev[9] = {};
    char *buf = nullptr;
    mms_status st = MMS_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking);
    for (int i = 0; i < 9 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    // staging: [in slab 0 | in slab 1 | out slab 0 | out slab 1], stream-ordered on the caller's stream
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&buf), 2 * (in_slab + out_slab), s);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "host sweep set-up");
    } else {
        cudaEvent_t start = ev[0], *in_ready = ev + 1, *in_free = ev + 3, *out_ready = ev + 5, *out_free = ev + 7;
        float *d_in[2] = {reinterpret_cast<float *>(buf), reinterpret_cast<float *>(buf + in_slab)};
        float *d_out[2] = {reinterpret_cast<float *>(buf + 2 * in_slab),
                           reinterpret_cast<float *>(buf + 2 * in_slab + out_slab)};
        // the copies start after everything queued on the caller's stream so far
        e = cudaEventRecord(start, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_in, start, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, start, 0);
        for (int64_t k = 0; k < nslab && e == cudaSuccess && st == MMS_OK; ++k) {
            const int b = (int)(k & 1);
            const int64_t z0 = k * tz, nzt = d->nz - z0 < tz ? d->nz - z0 : tz;
            const size_t ib = (size_t)((nzt + 2 * rz - 1) * ipz + (Y - 1) * ipy + X) * 4;
            if (k >= 2) e = cudaStreamWaitEvent(s_in, in_free[b], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_in[b], in + z0 * ipz, ib, cudaMemcpyHostToDevice, s_in);
            if (e == cudaSuccess) e = cudaEventRecord(in_ready[b], s_in);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, in_ready[b], 0);
            if (e == cudaSuccess && k >= 2) e = cudaStreamWaitEvent(s, out_free[b], 0);
            if (e != cudaSuccess) break;
            mms_stencil_desc sd = *d;
            sd.nz = nzt;
            sd.in_pitch_y = ipy;
            sd.in_pitch_z = ipz;
            sd.out_pitch_y = opy;
            sd.out_pitch_z = opz;
            st = apply(&sd, d_in[b], d_out[b], stream);
            if (st != MMS_OK) break;
            e = cudaEventRecord(in_free[b], s);
            if (e == cudaSuccess) e = cudaEventRecord(out_ready[b], s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, out_ready[b], 0);
            // rows of nx values only: the padding of the caller's pitched
            // output is not part of the result and is left untouched
            if (e == cudaSuccess) {
                const size_t w = (size_t)d->nx * 4, pitch = (size_t)opy * 4;
                if (opz == d->ny * opy) {
                    e = cudaMemcpy2DAsync(out + z0 * opz, pitch, d_out[b], pitch, w, (size_t)(nzt * d->ny),
                                          cudaMemcpyDeviceToHost, s_out);
                } else {
                    for (int64_t zz = 0; zz < nzt && e == cudaSuccess; ++zz)
                        e = cudaMemcpy2DAsync(out + (z0 + zz) * opz, pitch, d_out[b] + zz * opz, pitch, w,
                                              (size_t)d->ny, cudaMemcpyDeviceToHost, s_out);
                }
            }
            if (e == cudaSuccess) e = cudaEventRecord(out_free[b], s_out);
        }
        // the caller's stream takes over: it waits for the last copies, then
        // returns the staging memory to the pool
        cudaEvent_t done_in = ev[1], done_out = ev[5];
        cudaError_t j = cudaEventRecord(done_in, s_in);
        if (j == cudaSuccess) j = cudaStreamWaitEvent(s, done_in, 0);
        if (j == cudaSuccess) j = cudaEventRecord(done_out, s_out);
        if (j == cudaSuccess) j = cudaStreamWaitEvent(s, done_out, 0);
        cudaError_t f = cudaFreeAsync(buf, s);
        if (e == cudaSuccess) e = j;
        if (e == cudaSuccess) e = f;
        if (st == MMS_OK && e != cudaSuccess) st = cuda_fail(e, "host sweep pipeline");
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (s_in) cudaStreamDestroy(s_in);
    if (s_out) cudaStreamDestroy(s_out);
    return st;
}

}  // namespace mms

using namespace mms;

extern "C" {

mms_status mms_stencil_apply_host(const mms_stencil_desc *desc, const float *host_in, float *host_out,
                                  void *stream)
{
    return apply_host(desc, host_in, host_out, stream);
}

mms_status mms_stencil_apply(int shape, int radius, const float *coeffs, const float *in, float *out,
                             int64_t nx, int64_t ny, int64_t nz, void *stream)
{
    mms_stencil_desc d{};
    d.shape = shape;
    d.radius = radius;
    d.coeffs = coeffs;
    d.nx = nx;
    d.ny = ny;
    d.nz = nz;
    d.path = MMS_PATH_AUTO;
    d.variant = -1;
    return apply(&d, in, out, stream);
}

mms_status mms_stencil_apply_f64(const mms_stencil_desc *desc, const double *coeffs, const double *in, double *out,
                                 void *stream)
{
    return apply_f64(desc, coeffs, in, out, stream);
}

mms_status mms_stencil_apply_ex(const mms_stencil_desc *desc, const float *in, float *out, void *stream)
{
    return apply(desc, in, out, stream);
}

int32_t mms_num_variants(int shape, int radius, int path) { return num_variants(shape, radius, path); }

int32_t mms_auto_path(int shape, int radius, int tma_aligned)
{
    if (shape < MMS_STAR || shape > MMS_BOX2D || radius < 1 || radius > kMaxR) return -1;
    return auto_path(shape, radius, tma_aligned != 0);
}

int32_t mms_default_variant(int shape, int radius, int path, int64_t nx, int64_t ny, int64_t nz)
{
    (void)nx; (void)ny; (void)nz;
    if (num_variants(shape, radius, path) == 0) return -1;
    return default_variant(shape, radius, path);
}

mms_status mms_set_variant(int shape, int radius, int path, int32_t variant)
{
    if (shape < 0 || shape > 3 || radius < 1 || radius > kMaxR || path < 0 || path > MMS_PATH_NAIVE)
        return fail(MMS_E_ARG, "bad (shape, radius, path)");
    if (variant < -1 || variant >= num_variants(shape, radius, path))
        return fail(MMS_E_ARG, "variant %d out of range", variant);
    tuned_variant(shape, radius, path);  // initialises the table
    std::lock_guard<std::mutex> lk(g_var_mu);
    g_tuned[shape][radius][path] = variant >= 0 ? variant : kCleared;
    return MMS_OK;
}

const char *mms_last_error(void) { return g_last_error.c_str(); }

const char *mms_version(void) { return "mms-gb300 0.1 (sm_103a)"; }

mms_status mms_check_device(void *stream)
{
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
    unsigned *w = device_error_word();
    if (!w) return fail(MMS_E_CUDA, "device error word unavailable");
    unsigned h = 0;
    e = cudaMemcpy(&h, w, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read device error word");
    if (h) {
        const unsigned z = 0;
        cudaMemcpy(w, &z, sizeof z, cudaMemcpyHostToDevice);
    }
    if (h & kErrTimeout) return fail(MMS_E_TIMEOUT, "a bounded device-side wait ran out");
    if (h & kErrIndex) return fail(MMS_E_DEVICE, "a device-side index check failed");
    return MMS_OK;
}

}  // extern "C"

// ------------------------------------------------------------ wave ABI
namespace mms {

static mms_status wave_geo(const mms_wave_desc *d, const float *coeffs, WaveGeo *g)
{
    if (!d) return fail(MMS_E_ARG, "null wave descriptor");
    if (!coeffs) return fail(MMS_E_ARG, "null coefficient array");
    if (d->radius < 1 || d->radius > kMaxR) return fail(MMS_E_ARG, "radius %d outside 1..%d", d->radius, kMaxR);
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nx >= (1ll << 30) || d->ny >= (1ll << 30) || d->nz >= (1ll << 30))
        return fail(MMS_E_ARG, "interior sizes must be in 1..2^30");
    if (d->nshots < 1 || d->nshots > kMaxShots) return fail(MMS_E_ARG, "nshots %d outside 1..%d", d->nshots, kMaxShots);
    if (d->sponge_width < 0) return fail(MMS_E_ARG, "negative sponge width");
    if (d->rec_z < -1 || d->rec_z >= d->nz) return fail(MMS_E_ARG, "receiver plane %d outside the interior", d->rec_z);
    const int r = d->radius;
    const int64_t X = d->nx + 2 * r, Y = d->ny + 2 * r, Z = d->nz + 2 * r;
    g->nx = (int)d->nx; g->ny = (int)d->ny; g->nz = (int)d->nz; g->r = r; g->nshots = d->nshots;
    if (!resolve_pitches(X, Y, Z, d->pitch_y, d->pitch_z, &g->py, &g->pz))
        return fail(MMS_E_ARG, "field pitches not positive or spanning more than 2^46 elements");
    g->ss = d->shot_stride ? d->shot_stride : Z * g->pz;
    if (g->ss <= 0 || g->ss > kMaxSpan / d->nshots)
        return fail(MMS_E_ARG, "shot stride not positive or spanning more than 2^46 elements");
    if (g->py < X || g->pz < Y * g->py || g->ss < Z * g->pz) return fail(MMS_E_ARG, "field pitches below the padded extents");
    if (g->py % 4 || g->pz % 4 || g->ss % 4)
        return fail(MMS_E_ALIGN, "wave fields need pitches and shot stride that are multiples of 4 floats");
    g->sponge_w = d->sponge_width;
    g->sponge_a = d->sponge_a;
    g->rec_z = d->rec_z;
    g->gss = d->grad_shot_stride;
    if (g->gss > kMaxSpan / d->nshots)
        return fail(MMS_E_ARG, "gradient shot stride spans more than 2^46 elements");
    if (g->gss != 0 && g->gss < d->nx * d->ny * d->nz)
        return fail(MMS_E_ARG, "gradient shot stride %lld below the interior size", (long long)g->gss);
    for (int s = 0; s < d->nshots; ++s) {
        int x = -1, y = -1, z = -1;
        if (d->src_xyz) { x = d->src_xyz[3 * s]; y = d->src_xyz[3 * s + 1]; z = d->src_xyz[3 * s + 2]; }
        if (x >= 0 && (x >= d->nx || y < 0 || y >= d->ny || z < 0 || z >= d->nz))
            return fail(MMS_E_ARG, "source %d outside the interior", s);
        if (x < 0) x = y = z = -1;
        g->src[s][0] = x; g->src[s][1] = y; g->src[s][2] = z;
    }
    return MMS_OK;
}

static bool al16(const void *p) { return (reinterpret_cast<uintptr_t>(p) % 16) == 0; }

static size_t field_bytes(const WaveGeo &g) { return (size_t)g.nshots * g.ss * 4; }

// Extent of m (one padded field, shared by the shots).
static size_t model_bytes(const WaveGeo &g) { return (size_t)g.pz * (g.nz + 2 * g.r) * 4; }

// Extent of one step's receiver records (nshots x ny x nx floats).
static size_t rec_bytes(const WaveGeo &g) { return (size_t)g.nshots * g.ny * g.nx * 4; }

// Extent of the FP64 gradient: one interior, or one slice per shot.
static size_t grad_bytes(const WaveGeo &g)
{
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    return (size_t)(g.gss ? (g.nshots - 1) * g.gss + n : n) * 8;
}

// The records written by a step must not overlap anything it reads or writes.
static mms_status check_rec(const WaveGeo &g, const float *rec, const void *const *fields, int nf, const float *m)
{
    if (!rec || g.rec_z < 0) return MMS_OK;
    for (int i = 0; i < nf; ++i)
        if (overlaps(rec, rec_bytes(g), fields[i], field_bytes(g))) return fail(MMS_E_ARG, "rec overlaps a field");
    if (overlaps(rec, rec_bytes(g), m, model_bytes(g))) return fail(MMS_E_ARG, "rec overlaps m");
    return MMS_OK;
}

struct GraphEntry {
    uint64_t key;
    cudaGraphExec_t exec;
};
static std::mutex g_graph_mu;
static GraphEntry g_graphs[16];
static int g_ngraphs = 0;

static uint64_t mix(uint64_t h, uint64_t v) { return (h ^ v) * 0x100000001b3ull + (h >> 29); }

static uint64_t fbits(float f)
{
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
}

}  // namespace mms

extern "C" {

mms_status mms_wave_step(const mms_wave_desc *desc, const float *coeffs, const float *m, const float *p_cur,
                         float *p_prev, const float *src_amp, float *rec, void *stream)
{
    WaveGeo g{};
    mms_status st = wave_geo(desc, coeffs, &g);
    if (st != MMS_OK) return st;
    if (!m || !p_cur || !p_prev || !src_amp) return fail(MMS_E_ARG, "null field pointer");
    if (!al16(m) || !al16(p_cur) || !al16(p_prev)) return fail(MMS_E_ALIGN, "wave fields must be 16-byte aligned");
    if (overlaps(p_cur, field_bytes(g), p_prev, field_bytes(g))) return fail(MMS_E_ARG, "p_cur and p_prev overlap");
    if (overlaps(p_prev, field_bytes(g), m, model_bytes(g))) return fail(MMS_E_ARG, "an output field overlaps m");
    const void *fs[2] = {p_cur, p_prev};
    if ((st = check_rec(g, rec, fs, 2, m)) != MMS_OK) return st;
    cudaError_t e = launch_wave_fwd(g, coeffs, m, p_cur, p_prev, p_prev, src_amp, rec,
                                    reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "wave step launch");
}

mms_status mms_wave_step_to(const mms_wave_desc *desc, const float *coeffs, const float *m, const float *p_cur,
                            const float *p_prev, float *p_next, const float *src_amp, float *rec, void *stream)
{
    WaveGeo g{};
    mms_status st = wave_geo(desc, coeffs, &g);
    if (st != MMS_OK) return st;
    if (!m || !p_cur || !p_prev || !p_next || !src_amp) return fail(MMS_E_ARG, "null field pointer");
    if (!al16(m) || !al16(p_cur) || !al16(p_prev) || !al16(p_next))
        return fail(MMS_E_ALIGN, "wave fields must be 16-byte aligned");
    const size_t fb = field_bytes(g);
    if (overlaps(p_cur, fb, p_prev, fb)) return fail(MMS_E_ARG, "p_cur and p_prev overlap");
    if (overlaps(p_cur, fb, p_next, fb)) return fail(MMS_E_ARG, "p_cur and p_next overlap");
    if (p_next != p_prev && overlaps(p_prev, fb, p_next, fb))
        return fail(MMS_E_ARG, "p_prev and p_next overlap without being the same field");
    if (overlaps(p_next, fb, m, model_bytes(g))) return fail(MMS_E_ARG, "an output field overlaps m");
    const void *fs[3] = {p_cur, p_prev, p_next};
    if ((st = check_rec(g, rec, fs, 3, m)) != MMS_OK) return st;
    cudaError_t e = launch_wave_fwd(g, coeffs, m, p_cur, p_prev, p_next, src_amp, rec,
                                    reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "wave step launch");
}

mms_status mms_wave_forward(const mms_wave_desc *desc, const float *coeffs, const float *m, const float *amps,
                            int32_t nsteps, float *p0, float *p1, float *rec_all, float *ckpt, int32_t ckpt_every,
                            uint32_t flags, void *stream)
{
    WaveGeo g{};
    mms_status st = wave_geo(desc, coeffs, &g);
    if (st != MMS_OK) return st;
    if (nsteps < 0) return fail(MMS_E_ARG, "negative step count");
    if (!m || !amps || !p0 || !p1) return fail(MMS_E_ARG, "null field pointer");
    if (!al16(m) || !al16(p0) || !al16(p1)) return fail(MMS_E_ALIGN, "wave fields must be 16-byte aligned");
    if (overlaps(p0, field_bytes(g), p1, field_bytes(g))) return fail(MMS_E_ARG, "p0 and p1 overlap");
    if (ckpt && ckpt_every < 1) return fail(MMS_E_ARG, "checkpoint interval must be >= 1");
    if (rec_all && g.rec_z < 0) return fail(MMS_E_ARG, "records requested without a receiver plane");
    if (flags & ~MMS_WAVE_GRAPH) return fail(MMS_E_ARG, "unknown flags 0x%x", flags);
    if (nsteps == 0) return MMS_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t fb = field_bytes(g), mb = model_bytes(g);
    const int64_t rec_step = (int64_t)g.nshots * g.ny * g.nx;
    if (overlaps(p0, fb, m, mb) || overlaps(p1, fb, m, mb)) return fail(MMS_E_ARG, "a wavefield overlaps m");
    // checkpoint slots: one pair of fields for every ckpt_every steps
    const size_t cb = ckpt ? (size_t)((nsteps + ckpt_every - 1) / ckpt_every) * 2 * fb : 0;
    const size_t rb = rec_all ? (size_t)nsteps * rec_step * 4 : 0;
    if (ckpt && (overlaps(ckpt, cb, p0, fb) || overlaps(ckpt, cb, p1, fb) || overlaps(ckpt, cb, m, mb)))
        return fail(MMS_E_ARG, "ckpt overlaps a wavefield or m");
    if (rec_all && (overlaps(rec_all, rb, p0, fb) || overlaps(rec_all, rb, p1, fb) || overlaps(rec_all, rb, m, mb) ||
                    (ckpt && overlaps(rec_all, rb, ckpt, cb))))
        return fail(MMS_E_ARG, "rec_all overlaps a wavefield, m or ckpt");

    auto enqueue = [&]() -> mms_status {
        float *bufs[2] = {p0, p1};
        int c = 1;
        for (int n = 0; n < nsteps; ++n) {
            if (ckpt && n % ckpt_every == 0) {
                const int j = n / ckpt_every;
                char *slot = reinterpret_cast<char *>(ckpt) + (size_t)j * 2 * fb;
                cudaError_t e = cudaMemcpyAsync(slot, bufs[c], fb, cudaMemcpyDeviceToDevice, s);
                if (e == cudaSuccess) e = cudaMemcpyAsync(slot + fb, bufs[1 - c], fb, cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) return cuda_fail(e, "checkpoint copy");
            }
            cudaError_t e = launch_wave_fwd(g, coeffs, m, bufs[c], bufs[1 - c], bufs[1 - c],
                                            amps + (int64_t)n * g.nshots,
                                            rec_all ? rec_all + n * rec_step : nullptr, s);
            if (e != cudaSuccess) return cuda_fail(e, "wave step launch");
            c = 1 - c;
        }
        return MMS_OK;
    };
    if (!(flags & MMS_WAVE_GRAPH)) return enqueue();

    // Key of the captured sequence: every argument that ends up in a node.
    uint64_t key = 0xcbf29ce484222325ull;
    const uint64_t vals[] = {(uint64_t)(uintptr_t)m, (uint64_t)(uintptr_t)amps, (uint64_t)nsteps,
                             (uint64_t)(uintptr_t)p0, (uint64_t)(uintptr_t)p1, (uint64_t)(uintptr_t)rec_all,
                             (uint64_t)(uintptr_t)ckpt, (uint64_t)ckpt_every, (uint64_t)g.nx, (uint64_t)g.ny,
                             (uint64_t)g.nz, (uint64_t)g.r, (uint64_t)g.nshots, (uint64_t)g.py, (uint64_t)g.pz,
                             (uint64_t)g.ss, (uint64_t)g.sponge_w, fbits(g.sponge_a),
                             (uint64_t)(int64_t)g.rec_z};
    for (uint64_t v : vals) key = mix(key, v);
    for (int i = 0; i < 3 * (2 * g.r + 1); ++i) key = mix(key, fbits(coeffs[i]));
    for (int i = 0; i < g.nshots; ++i)
        key = mix(key, ((uint64_t)(uint32_t)g.src[i][0] << 40) ^ ((uint64_t)(uint32_t)g.src[i][1] << 20) ^
                           (uint32_t)g.src[i][2]);
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (int i = 0; i < g_ngraphs; ++i)
        if (g_graphs[i].key == key) {
            cudaError_t e = cudaGraphLaunch(g_graphs[i].exec, s);
            return e == cudaSuccess ? MMS_OK : cuda_fail(e, "graph launch");
        }
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaStreamDestroy(cap); return cuda_fail(e, "begin capture"); }
    cudaStream_t saved = s;
    s = cap;
    mms_status qs = enqueue();
    s = saved;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (qs != MMS_OK) { if (graph) cudaGraphDestroy(graph); return qs; }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    if (g_ngraphs == 16) {
        // Oldest entry out; a replay of it may still be running, so wait for
        // the device before destroying it.
        cudaDeviceSynchronize();
        cudaGraphExecDestroy(g_graphs[0].exec);
        for (int i = 1; i < 16; ++i) g_graphs[i - 1] = g_graphs[i];
        g_ngraphs = 15;
    }
    g_graphs[g_ngraphs++] = {key, exec};
    e = cudaGraphLaunch(exec, s);
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "graph launch");
}

static mms_status wave_adjoint(const mms_wave_desc *desc, const float *coeffs, const float *m, const float *lam_cur,
                               float *lam_prev, const float *resid, const float *a_n, double *grad_m, void *stream,
                               bool lapin)
{
    WaveGeo g{};
    mms_status st = wave_geo(desc, coeffs, &g);
    if (st != MMS_OK) return st;
    if (!m || !lam_cur || !lam_prev) return fail(MMS_E_ARG, "null field pointer");
    if (a_n && !grad_m) return fail(MMS_E_ARG, "a_n given without grad_m");
    if (resid && g.rec_z < 0) return fail(MMS_E_ARG, "residual given without a receiver plane");
    if (!al16(m) || !al16(lam_cur) || !al16(lam_prev) || (a_n && !al16(a_n)))
        return fail(MMS_E_ALIGN, "wave fields must be 16-byte aligned");
    if (overlaps(lam_cur, field_bytes(g), lam_prev, field_bytes(g))) return fail(MMS_E_ARG, "lam_cur and lam_prev overlap");
    if (a_n && overlaps(a_n, field_bytes(g), lam_prev, field_bytes(g))) return fail(MMS_E_ARG, "a_n and lam_prev overlap");
    if (overlaps(lam_prev, field_bytes(g), m, model_bytes(g))) return fail(MMS_E_ARG, "lam_prev overlaps m");
    if (resid && overlaps(resid, rec_bytes(g), lam_prev, field_bytes(g))) return fail(MMS_E_ARG, "resid overlaps lam_prev");
    if (grad_m) {
        const size_t gb = grad_bytes(g), fb = field_bytes(g);
        if (overlaps(grad_m, gb, m, model_bytes(g)) || overlaps(grad_m, gb, lam_cur, fb) ||
            overlaps(grad_m, gb, lam_prev, fb) || (a_n && overlaps(grad_m, gb, a_n, fb)) ||
            (resid && overlaps(grad_m, gb, resid, rec_bytes(g))))
            return fail(MMS_E_ARG, "grad_m overlaps a field");
    }
    cudaError_t e = launch_wave_adj(g, coeffs, m, lam_cur, lam_prev, resid, a_n, grad_m,
                                    reinterpret_cast<cudaStream_t>(stream), lapin);
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "adjoint step launch");
}

mms_status mms_wave_adjoint(const mms_wave_desc *desc, const float *coeffs, const float *m, const float *lam_cur,
                            float *lam_prev, const float *resid, const float *a_n, double *grad_m, void *stream)
{
    return wave_adjoint(desc, coeffs, m, lam_cur, lam_prev, resid, a_n, grad_m, stream, false);
}

mms_status mms_wave_adjoint_lap(const mms_wave_desc *desc, const float *coeffs, const float *m, const float *lam_cur,
                                float *lam_prev, const float *resid, const float *lap_a, double *grad_m, void *stream)
{
    return wave_adjoint(desc, coeffs, m, lam_cur, lam_prev, resid, lap_a, grad_m, stream, true);
}

mms_status mms_wave_adjoint_scaled(const mms_wave_desc *desc, const float *coeffs, const float *m,
                                   const float *mu_cur, float *mu_prev, const float *resid, const float *lap_a,
                                   double *grad_m, void *stream)
{
    WaveGeo g{};
    mms_status st = wave_geo(desc, coeffs, &g);
    if (st != MMS_OK) return st;
    if (!m || !mu_cur || !mu_prev) return fail(MMS_E_ARG, "null field pointer");
    if (lap_a && !grad_m) return fail(MMS_E_ARG, "lap_a given without grad_m");
    if (resid && g.rec_z < 0) return fail(MMS_E_ARG, "residual given without a receiver plane");
    if (!al16(m) || !al16(mu_cur) || !al16(mu_prev) || (lap_a && !al16(lap_a)))
        return fail(MMS_E_ALIGN, "wave fields must be 16-byte aligned");
    const size_t fb = field_bytes(g);
    if (overlaps(mu_cur, fb, mu_prev, fb)) return fail(MMS_E_ARG, "mu_cur and mu_prev overlap");
    if (lap_a && overlaps(lap_a, fb, mu_prev, fb)) return fail(MMS_E_ARG, "lap_a and mu_prev overlap");
    if (overlaps(mu_prev, fb, m, model_bytes(g))) return fail(MMS_E_ARG, "mu_prev overlaps m");
    if (resid && overlaps(resid, rec_bytes(g), mu_prev, fb)) return fail(MMS_E_ARG, "resid overlaps mu_prev");
    if (grad_m) {
        const size_t gb = grad_bytes(g);
        if (overlaps(grad_m, gb, m, model_bytes(g)) || overlaps(grad_m, gb, mu_cur, fb) ||
            overlaps(grad_m, gb, mu_prev, fb) || (lap_a && overlaps(grad_m, gb, lap_a, fb)) ||
            (resid && overlaps(grad_m, gb, resid, rec_bytes(g))))
            return fail(MMS_E_ARG, "grad_m overlaps a field");
    }
    cudaError_t e = launch_wave_adj_scaled(g, coeffs, m, mu_cur, mu_prev, resid, lap_a, grad_m,
                                           reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "scaled adjoint step launch");
}

mms_status mms_grad_divide_m(const mms_wave_desc *desc, const float *m, double *grad_m, void *stream)
{
    WaveGeo g{};
    static const float dummy[27] = {0};
    mms_status st = wave_geo(desc, dummy, &g);
    if (st != MMS_OK) return st;
    if (!m || !grad_m) return fail(MMS_E_ARG, "null pointer");
    if (overlaps(grad_m, (size_t)g.nx * g.ny * g.nz * 8, m, model_bytes(g))) return fail(MMS_E_ARG, "grad_m overlaps m");
    cudaError_t e = launch_grad_divide_m(g, m, grad_m, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "divide-by-m kernel launch");
}

mms_status mms_wave_step_lap(const mms_wave_desc *desc, const float *coeffs, const float *m, const float *p_cur,
                             const float *p_prev, float *p_next, float *lap_out, const float *src_amp, float *rec,
                             void *stream)
{
    WaveGeo g{};
    mms_status st = wave_geo(desc, coeffs, &g);
    if (st != MMS_OK) return st;
    if (!m || !p_cur || !p_prev || !p_next || !lap_out || !src_amp) return fail(MMS_E_ARG, "null field pointer");
    if (!al16(m) || !al16(p_cur) || !al16(p_prev) || !al16(p_next) || !al16(lap_out))
        return fail(MMS_E_ALIGN, "wave fields must be 16-byte aligned");
    const size_t fb = field_bytes(g);
    if (overlaps(p_cur, fb, p_prev, fb)) return fail(MMS_E_ARG, "p_cur and p_prev overlap");
    if (overlaps(p_cur, fb, p_next, fb)) return fail(MMS_E_ARG, "p_cur and p_next overlap");
    if (p_next != p_prev && overlaps(p_prev, fb, p_next, fb))
        return fail(MMS_E_ARG, "p_prev and p_next overlap without being the same field");
    const void *others[3] = {p_cur, p_prev, p_next};
    for (const void *q : others)
        if (overlaps(lap_out, fb, q, fb)) return fail(MMS_E_ARG, "lap_out overlaps a field");
    if (overlaps(lap_out, fb, m, (size_t)g.pz * (g.nz + 2 * g.r) * 4) ||
        overlaps(p_next, fb, m, (size_t)g.pz * (g.nz + 2 * g.r) * 4))
        return fail(MMS_E_ARG, "an output field overlaps m");
    cudaError_t e = launch_wave_fwd(g, coeffs, m, p_cur, p_prev, p_next, src_amp, rec,
                                    reinterpret_cast<cudaStream_t>(stream), lap_out);
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "wave step launch");
}

mms_status mms_vti_model(const mms_wave_desc *desc, const float *vp, const float *eps, const float *delta,
                         float *mv, float *rho, float dt, float h, void *stream)
{
    WaveGeo g{};
    static const float dummy[27] = {0};
    mms_status st = wave_geo(desc, dummy, &g);
    if (st != MMS_OK) return st;
    if (!vp || !eps || !delta || !mv || !rho) return fail(MMS_E_ARG, "null pointer");
    if (!(dt > 0.f) || !(h > 0.f)) return fail(MMS_E_ARG, "dt and h must be positive");
    const size_t mb = (size_t)g.pz * (g.nz + 2 * g.r) * 4;
    const size_t nb = (size_t)g.nx * g.ny * g.nz * 4;
    if (overlaps(mv, mb, rho, mb)) return fail(MMS_E_ARG, "mv and rho overlap");
    const float *ins[3] = {vp, eps, delta};
    for (const float *q : ins)
        if (overlaps(q, nb, mv, mb) || overlaps(q, nb, rho, mb)) return fail(MMS_E_ARG, "mv or rho overlaps an input");
    cudaError_t e = launch_vti_model(g, vp, eps, delta, mv, rho, dt, h, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "VTI model kernel launch");
}

mms_status mms_vti_step(const mms_wave_desc *desc, const float *coeffs, const float *mv, const float *rho,
                        const float *sh_cur, const float *sv_cur, const float *sh_prev, const float *sv_prev,
                        float *sh_next, float *sv_next, const float *src_amp, float *rec, void *stream)
{
    WaveGeo g{};
    mms_status st = wave_geo(desc, coeffs, &g);
    if (st != MMS_OK) return st;
    if (!mv || !rho || !sh_cur || !sv_cur || !sh_prev || !sv_prev || !sh_next || !sv_next || !src_amp)
        return fail(MMS_E_ARG, "null field pointer");
    const void *all[8] = {mv, rho, sh_cur, sv_cur, sh_prev, sv_prev, sh_next, sv_next};
    for (const void *q : all)
        if (!al16(q)) return fail(MMS_E_ALIGN, "VTI fields must be 16-byte aligned");
    const size_t fb = field_bytes(g);
    const float *rd[4] = {sh_cur, sv_cur, sh_prev, sv_prev};
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b)
            if (overlaps(rd[a], fb, rd[b], fb)) return fail(MMS_E_ARG, "VTI input fields %d and %d overlap", a, b);
    if (overlaps(sh_next, fb, sv_next, fb)) return fail(MMS_E_ARG, "sh_next and sv_next overlap");
    const size_t mb = (size_t)g.pz * (g.nz + 2 * g.r) * 4;
    if (overlaps(sh_next, fb, mv, mb) || overlaps(sh_next, fb, rho, mb) || overlaps(sv_next, fb, mv, mb) ||
        overlaps(sv_next, fb, rho, mb))
        return fail(MMS_E_ARG, "an output field overlaps the medium");
    const float *nx2[2] = {sh_next, sv_next};
    for (int o = 0; o < 2; ++o)
        for (int a = 0; a < 4; ++a) {
            if (a == 2 + o && nx2[o] == rd[a]) continue;  // in place over the matching previous state
            if (overlaps(nx2[o], fb, rd[a], fb))
                return fail(MMS_E_ARG, "%s overlaps an input field other than its own previous state",
                            o ? "sv_next" : "sh_next");
        }
    cudaError_t e = launch_vti_step(g, coeffs, mv, rho, sh_cur, sv_cur, sh_prev, sv_prev, sh_next, sv_next, src_amp,
                                    rec, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "VTI step launch");
}

mms_status mms_tti_model(const mms_wave_desc *desc, const float *vp, const float *vs, const float *eps,
                         const float *delta, const float *alpha, const float *theta, const float *phi,
                         float *med, float dt, float h, void *stream)
{
    WaveGeo g{};
    static const float dummy[27] = {0};
    mms_status st = wave_geo(desc, dummy, &g);
    if (st != MMS_OK) return st;
    if (!vp || !vs || !eps || !delta || !alpha || !theta || !phi || !med) return fail(MMS_E_ARG, "null pointer");
    if (!(dt > 0.f) || !(h > 0.f)) return fail(MMS_E_ARG, "dt and h must be positive");
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    const float *ins[7] = {vp, vs, eps, delta, alpha, theta, phi};
    for (const float *q : ins)
        if (overlaps(q, (size_t)n * 4, med, (size_t)n * 32)) return fail(MMS_E_ARG, "med overlaps an input");
    cudaError_t e = launch_tti_model(n, vp, vs, eps, delta, alpha, theta, phi, med, dt, h,
                                     reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "TTI model kernel launch");
}

mms_status mms_tti_step(const mms_wave_desc *desc, const float *w2, const float *w1, const float *med,
                        const float *p_cur, const float *q_cur, const float *p_prev, const float *q_prev,
                        float *p_next, float *q_next, float *work, const float *src_amp, float *rec, void *stream)
{
    WaveGeo g{};
    static const float dummy[27] = {0};
    mms_status st = wave_geo(desc, dummy, &g);
    if (st != MMS_OK) return st;
    if (!w2 || !w1) return fail(MMS_E_ARG, "null weight array");
    if (!med || !p_cur || !q_cur || !p_prev || !q_prev || !p_next || !q_next || !work || !src_amp)
        return fail(MMS_E_ARG, "null field pointer");
    const void *al[9] = {med, p_cur, q_cur, p_prev, q_prev, p_next, q_next, work, nullptr};
    for (int i = 0; i < 8; ++i)
        if (!al16(al[i])) return fail(MMS_E_ALIGN, "TTI fields and work must be 16-byte aligned");
    const size_t fb = field_bytes(g);
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    const size_t wb = (size_t)4 * g.nshots * n * 4;
    const float *rd[4] = {p_cur, q_cur, p_prev, q_prev};
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b)
            if (overlaps(rd[a], fb, rd[b], fb)) return fail(MMS_E_ARG, "TTI input fields %d and %d overlap", a, b);
    if (overlaps(p_next, fb, q_next, fb)) return fail(MMS_E_ARG, "p_next and q_next overlap");
    const float *nx2[2] = {p_next, q_next};
    for (int o = 0; o < 2; ++o) {
        for (int a = 0; a < 4; ++a) {
            if (a == 2 + o && nx2[o] == rd[a]) continue;
            if (overlaps(nx2[o], fb, rd[a], fb))
                return fail(MMS_E_ARG, "%s overlaps an input field other than its own previous state",
                            o ? "q_next" : "p_next");
        }
        if (overlaps(nx2[o], fb, work, wb)) return fail(MMS_E_ARG, "work overlaps an output field");
        if (overlaps(nx2[o], fb, med, (size_t)n * 32)) return fail(MMS_E_ARG, "an output field overlaps med");
    }
    for (int a = 0; a < 4; ++a)
        if (overlaps(rd[a], fb, work, wb)) return fail(MMS_E_ARG, "work overlaps an input field");
    if (overlaps(med, (size_t)n * 32, work, wb)) return fail(MMS_E_ARG, "work overlaps med");
    cudaError_t e = launch_tti_step(g, w2, w1, med, p_cur, q_cur, p_prev, q_prev, p_next, q_next, work, src_amp, rec,
                                    reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "TTI step launch");
}

int32_t mms_aniso_num_variants(int32_t kind) { return kind == 0 ? vti_num_variants() : 0; }

mms_status mms_aniso_set_variant(int32_t kind, int32_t variant)
{
    if (kind != 0) return fail(MMS_E_ARG, "unknown anisotropic kind %d", kind);
    if (!vti_set_variant(variant)) return fail(MMS_E_ARG, "variant %d outside 0..%d", variant, vti_num_variants() - 1);
    return MMS_OK;
}

mms_status mms_model_from_velocity(const mms_wave_desc *desc, const float *v, float *m, float dt, float h,
                                   void *stream)
{
    WaveGeo g{};
    static const float dummy[27] = {0};
    mms_status st = wave_geo(desc, dummy, &g);
    if (st != MMS_OK) return st;
    if (!v || !m) return fail(MMS_E_ARG, "null pointer");
    if (!(dt > 0.f) || !(h > 0.f)) return fail(MMS_E_ARG, "dt and h must be positive");
    if (overlaps(v, (size_t)g.nx * g.ny * g.nz * 4, m, model_bytes(g))) return fail(MMS_E_ARG, "m overlaps v");
    cudaError_t e = launch_model_from_velocity(g, v, m, dt, h, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "model kernel launch");
}

mms_status mms_grad_to_velocity(const double *grad_m, const float *v, double *grad_v, int64_t n, float dt, float h,
                                void *stream)
{
    if (n < 0) return fail(MMS_E_ARG, "negative length");
    if (n == 0) return MMS_OK;
    if (!grad_m || !v || !grad_v) return fail(MMS_E_ARG, "null pointer");
    if (!(dt > 0.f) || !(h > 0.f)) return fail(MMS_E_ARG, "dt and h must be positive");
    // element-wise: grad_v may be grad_m itself, but not a shifted copy of it
    if (grad_v != grad_m && overlaps(grad_v, (size_t)n * 8, grad_m, (size_t)n * 8))
        return fail(MMS_E_ARG, "grad_v overlaps grad_m without being it");
    if (overlaps(grad_v, (size_t)n * 8, v, (size_t)n * 4)) return fail(MMS_E_ARG, "grad_v overlaps v");
    cudaError_t e = launch_grad_to_velocity(grad_m, v, grad_v, n, dt, h, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "chain-rule kernel launch");
}

mms_status mms_sum_f64(const double *slices, int32_t nslices, int64_t stride, int64_t n, double *out,
                       void *stream)
{
    if (n < 0) return fail(MMS_E_ARG, "negative length");
    if (nslices < 1) return fail(MMS_E_ARG, "nslices %d below 1", nslices);
    if (n > kMaxSpan || (nslices > 1 && stride > kMaxSpan / nslices))
        return fail(MMS_E_ARG, "slices spanning more than 2^46 elements");
    if (nslices > 1 && stride < n) return fail(MMS_E_ARG, "slice stride %lld below the length", (long long)stride);
    if (n == 0) return MMS_OK;
    if (!slices || !out) return fail(MMS_E_ARG, "null pointer");
    for (int s = 1; s < nslices; ++s)
        if (overlaps(out, (size_t)n * 8, slices + (int64_t)s * stride, (size_t)n * 8))
            return fail(MMS_E_ARG, "out overlaps slice %d", s);
    if (out != slices && overlaps(out, (size_t)n * 8, slices, (size_t)n * 8))
        return fail(MMS_E_ARG, "out overlaps the first slice without being it");
    cudaError_t e = launch_sum_f64(slices, nslices, stride, n, out, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "sum kernel launch");
}

mms_status mms_selftest_timeout(uint32_t limit_us, void *stream)
{
    if (limit_us < 1 || limit_us > 2000000) return fail(MMS_E_ARG, "limit %u us outside 1..2000000", limit_us);
    cudaError_t e = launch_wait_selftest((unsigned long long)limit_us * 1000ull, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "self-test launch");
}

mms_status mms_dot_f64(const float *a, const float *b, int64_t n, double *result, void *stream)
{
    if (n < 0) return fail(MMS_E_ARG, "negative length");
    if (!result) return fail(MMS_E_ARG, "null result pointer");
    if (n > 0 && (!a || !b)) return fail(MMS_E_ARG, "null input pointer");
    if (n > 0 && (overlaps(result, 8, a, (size_t)n * 4) || overlaps(result, 8, b, (size_t)n * 4)))
        return fail(MMS_E_ARG, "result overlaps an input");
    cudaError_t e = launch_dot_f64(a, b, n, result, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "dot kernel launch");
}

}  // extern "C"
