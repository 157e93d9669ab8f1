// noalloc.cu -- the star sweep on tensor cores for callers that cannot
// allocate device memory (mms_stencil_apply_noalloc in include/mms.h).
//
// The paper's two-pass form of the star (Sec. 4.3) needs a temporary grid
// of nx*ny*nz floats for the in-plane partial sums.  mms_stencil_apply_ex
// takes it from the device's stream-ordered memory pool on every call; some
// callers cannot allow that: code whose memory is budgeted up front (a host
// that reserves all device memory for its own allocator), code that may not
// call cudaMalloc-family routines at all (a driver or plugin with a fixed
// footprint).  Here the temporary grid is a file-scope device array of a
// fixed size, part of the library's own module, so the call allocates
// nothing.
#include "common.cuh"
#include "validate.cuh"

namespace mms {

mms_status fail(mms_status st, const char *fmt, ...);
mms_status cuda_fail(cudaError_t e, const char *what);
// band_tc.cu: the two-pass star variant with the tile shape of variant v
int band_tc_two_pass_variant(int v);

namespace {

// The temporary grid.  Every device that loads this module holds these
// MMS_NOALLOC_MAX_POINTS floats (32 MiB) until the process exits.
static __device__ __align__(256) float g_noalloc_scratch[MMS_NOALLOC_MAX_POINTS];

// Device address of g_noalloc_scratch in the calling thread's current
// context.  In host code the array's name only stands for the symbol.  The
// address is looked up on every call (a host-side query): a cached one
// would go stale when the context changes under the same device number
// (after cudaDeviceReset the module is loaded again, possibly elsewhere; a
// caller's own driver-API context has its own copy of the array).
mms_status scratch_of_current_context(float **ptr)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-alloc scratch");
    *ptr = static_cast<float *>(p);
    return MMS_OK;
}

bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + nb && b0 < a0 + na;
}

}  // namespace

static mms_status apply_noalloc(const mms_stencil_desc *d, const float *in, float *out, void *stream)
{
    if (!d) return fail(MMS_E_ARG, "null descriptor");
    const int r = d->radius;
    if (d->shape != MMS_STAR) return fail(MMS_E_UNSUPPORTED, "the no-alloc sweep is the star shape only");
    if (r < 1 || r > kMaxR) return fail(MMS_E_ARG, "radius %d outside 1..%d", r, kMaxR);
    if (!d->coeffs) return fail(MMS_E_ARG, "null coefficient array");
    if (d->nx < 0 || d->ny < 0 || d->nz < 0) return fail(MMS_E_ARG, "negative size");
    if (d->nx >= (1ll << 30) || d->ny >= (1ll << 30) || d->nz >= (1ll << 30))
        return fail(MMS_E_ARG, "size above 2^30");
    if (d->path < MMS_PATH_AUTO || d->path > MMS_PATH_NAIVE) return fail(MMS_E_ARG, "unknown path %d", d->path);
    int path = d->path == MMS_PATH_AUTO ? MMS_PATH_BF16X3 : d->path;
    if (path != MMS_PATH_TF32 && path != MMS_PATH_3XTF32 && path != MMS_PATH_BF16X3)
        return fail(MMS_E_UNSUPPORTED, "the no-alloc sweep runs on tensor-core paths only (path %d)", d->path);
    if (d->variant < -1) return fail(MMS_E_ARG, "variant %d", d->variant);
    if (d->nx == 0 || d->ny == 0 || d->nz == 0) return MMS_OK;
    // nx*ny*nz <= limit, compared by division (the product of sizes up to
    // 2^30 each does not fit 64 bits)
    if (d->nx > (int64_t)MMS_NOALLOC_MAX_POINTS / d->ny / d->nz)
        return fail(MMS_E_ARG, "interior of %lld x %lld x %lld points is above the no-alloc limit of %lld points",
                    (long long)d->nx, (long long)d->ny, (long long)d->nz, (long long)MMS_NOALLOC_MAX_POINTS);
    if (!in || !out) return fail(MMS_E_ARG, "null grid pointer");
    const int64_t X = d->nx + 2 * r, Y = d->ny + 2 * r, Z = d->nz + 2 * r;
    int64_t ipy, ipz, opy, opz;
    if (!resolve_pitches(X, Y, Z, d->in_pitch_y, d->in_pitch_z, &ipy, &ipz) ||
        !resolve_pitches(d->nx, d->ny, d->nz, d->out_pitch_y, d->out_pitch_z, &opy, &opz))
        return fail(MMS_E_ARG, "pitches not positive or spanning more than 2^46 elements");
    if (ipy < X || ipz < Y * ipy)
        return fail(MMS_E_ARG, "input pitches (%lld, %lld) below the padded extents", (long long)ipy, (long long)ipz);
    if (opy < d->nx || opz < d->ny * opy)
        return fail(MMS_E_ARG, "output pitches (%lld, %lld) below the interior extents", (long long)opy,
                    (long long)opz);
    const size_t in_bytes = (size_t)((Z - 1) * ipz + (Y - 1) * ipy + X) * 4;
    const size_t out_bytes = (size_t)((d->nz - 1) * opz + (d->ny - 1) * opy + d->nx) * 4;
    if (ranges_overlap(in, in_bytes, out, out_bytes)) return fail(MMS_E_ARG, "input and output overlap");
    if ((reinterpret_cast<uintptr_t>(in) % 16) != 0 || (ipy % 4) != 0 || (ipz % 4) != 0)
        return fail(MMS_E_ALIGN, "TMA path needs a 16-byte aligned input and pitches that are multiples of 4 floats");
    if (!band_tc_supported(MMS_STAR, r, path))
        return fail(MMS_E_UNSUPPORTED, "path %d does not support the star of radius %d", path, r);
    // the two-pass form with the tile shape of the requested (or the
    // library's default) variant: the form that needs the temporary grid
    const int nvar = band_tc_variants(MMS_STAR, r, path);
    if (d->variant >= nvar) return fail(MMS_E_ARG, "variant %d of %d", d->variant, nvar);
    const int v = band_tc_two_pass_variant(
        d->variant >= 0 ? d->variant : mms_default_variant(MMS_STAR, r, path, d->nx, d->ny, d->nz));

    float *scratch = nullptr;
    mms_status st = scratch_of_current_context(&scratch);
    if (st != MMS_OK) return st;

    Sweep s{MMS_STAR, r, d->nx, d->ny, d->nz, in, ipy, ipz, out, opy, opz, d->coeffs, v,
            reinterpret_cast<cudaStream_t>(stream)};
    int bx, by, bz, swz;
    band_tc_box(MMS_STAR, r, path, v, &bx, &by, &bz, &swz);
    CUtensorMap map;
    if (!encode_tmap_3d(&map, in, X, Y, Z, ipy, ipz, bx, by, bz, swz != 0))
        return fail(MMS_E_CUDA, "cuTensorMapEncodeTiled refused the input grid");
    // The planar pass writes every element of the first nx*ny*nz floats of
    // the array before the z pass reads it, so nothing needs clearing.
    cudaError_t e = launch_band_tc(s, path, map, v, scratch);
    return e == cudaSuccess ? MMS_OK : cuda_fail(e, "no-alloc tensor-core star launch");
}

}  // namespace mms

extern "C" mms_status mms_stencil_apply_noalloc(const mms_stencil_desc *desc, const float *in, float *out,
                                                void *stream)
{
    return mms::apply_noalloc(desc, in, out, stream);
}
