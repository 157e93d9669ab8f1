/*
 * mms.h -- C ABI of the GB300 (sm_103a) stencil-as-matrix-product library.
 *
 * All entry points are plain C: pointers, sizes and enums, no C++ or torch
 * types.  Device pointers are CUDA global-memory addresses of the calling
 * thread's current device; host pointers are ordinary process memory.
 * `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 * stream).  Every call is asynchronous on `stream` unless stated otherwise.
 *
 * Ownership: the caller owns every buffer.  Host arrays (coefficients,
 * source positions, descriptors) are read before the call returns and may be
 * freed right after.  Device buffers must stay valid until the work queued
 * on `stream` has finished.  The library keeps only caches keyed by value
 * (prepared coefficient bands, tensor maps) and one device error word.
 *
 * Errors: arguments are validated before anything is queued.  A non-OK
 * status means nothing was queued by that call (MMS_E_CUDA: a launch was
 * refused by the runtime); mms_last_error() returns a thread-local message.
 * Device-side faults of the library's own checks (a bounded wait that ran
 * out, an index check in a debug build) set a device error word that
 * mms_check_device() reads and clears; no kernel traps.
 *
 * Grid conventions (paper Sec. 1, Fig. 1 and Sec. 4.1): the interior has
 * nx*ny*nz points, x fastest.  A stencil of radius r reads a grid padded by
 * r on every face: padded element (X,Y,Z), 0 <= X < nx+2r etc., lives at
 * in[Z*in_pitch_z + Y*in_pitch_y + X].  Output point (x,y,z) lives at
 * out[z*out_pitch_z + y*out_pitch_y + x] and is
 *     out(x,y,z) = sum_d c_d * in(x+r+dx, y+r+dy, z+r+dz)
 * over the stencil's offsets d.  Pitches are in elements; 0 selects the
 * dense value (in: nx+2r and (ny+2r)*pitch_y; out: nx and ny*pitch_y).
 * Sizes are below 2^30 per axis; a pitch or stride that is negative, or
 * that spans more than 2^46 elements (rows * pitch_y, planes * pitch_z,
 * shots * shot_stride), is refused with MMS_E_ARG before any extent is
 * computed from it.
 */
#ifndef MMS_H
#define MMS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MMS_OK = 0,
    MMS_E_ARG = 1,          /* invalid argument (radius, sizes, null or overlapping buffers) */
    MMS_E_UNSUPPORTED = 2,  /* valid request that this build does not implement */
    MMS_E_ALIGN = 3,        /* a pitch or address that the forced path cannot use */
    MMS_E_CUDA = 4,         /* the CUDA runtime refused a call or launch */
    MMS_E_TIMEOUT = 5,      /* a bounded device-side wait ran out (from mms_check_device) */
    MMS_E_DEVICE = 6,       /* a device-side check failed (from mms_check_device) */
    MMS_E_NOMEM = 7         /* host-side allocation of a cache entry failed */
} mms_status;

/* Stencil shapes (paper Sec. 1, Fig. 1; Table I lists 3D and 2D kernels). */
typedef enum {
    MMS_STAR = 0,    /* axis neighbours only: 6r+1 points */
    MMS_BOX = 1,     /* full (2r+1)^3 cube */
    MMS_STAR2D = 2,  /* planar star, x and y neighbours: 4r+1 points per plane */
    MMS_BOX2D = 3    /* planar box, (2r+1)^2 points per plane */
} mms_shape;

/* Computation paths of a sweep. */
typedef enum {
    MMS_PATH_AUTO = 0,       /* library choice: the tuned path meeting FP32-level accuracy (mms_auto_path) */
    MMS_PATH_CUDA_CORE = 1,  /* FP32 FMA on CUDA cores, TMA-staged plane tiles */
    MMS_PATH_TF32 = 2,       /* tensor cores, one TF32 product (reduced accuracy) */
    MMS_PATH_3XTF32 = 3,     /* tensor cores, TF32 hi/lo split, 3 products, FP32 accumulate */
    MMS_PATH_BF16X3 = 4,     /* tensor cores, BF16 hi/lo split, 3 products, FP32 accumulate */
    MMS_PATH_NAIVE = 5       /* one thread per point, global loads (any pitch) */
} mms_path;

/*
 * Coefficient layouts (host, float32):
 *   star: 3*(2r+1) values, c[axis*(2r+1) + d+r] for axis 0=x, 1=y, 2=z and
 *         d = -r..r; the applied centre weight is cx[0]+cy[0]+cz[0];
 *   box:  (2r+1)^3 values, c[((dz+r)*(2r+1) + dy+r)*(2r+1) + dx+r].
 *   star2d: 2*(2r+1) values, c[axis*(2r+1) + d+r] for axis 0=x, 1=y; the
 *         applied centre is cx[0]+cy[0];
 *   box2d:  (2r+1)^2 values, c[(dy+r)*(2r+1) + dx+r].
 * The paper's Sec. 4.1 turns each axis's 1D weights into a banded coefficient
 * matrix; the library builds those bands from these arrays.
 *
 * The planar shapes (Table I's 2D kernels) apply to nz independent planes
 * padded by r in x and y only: input element (X,Y,z), 0 <= X < nx+2r,
 * 0 <= Y < ny+2r, 0 <= z < nz, lives at in[z*in_pitch_z + Y*in_pitch_y + X]
 * (dense in_pitch_z = (ny+2r)*in_pitch_y) and
 *     out(x,y,z) = sum_d c_d * in(x+r+dx, y+r+dy, z);
 * nz = 1 is a single 2D grid.
 */

/*
 * One stencil sweep with dense layouts (pitches 0) and the AUTO path.
 * shape: MMS_STAR or MMS_BOX; radius: 1..4; coeffs: host, layout above;
 * in: device, (nz+2r)(ny+2r)(nx+2r) floats; out: device, nz*ny*nx floats;
 * in and out must not overlap.  nx, ny, nz >= 0 (an empty interior queues
 * nothing and returns MMS_OK).
 * Defined by: paper Sec. 1 (star and box stencils, Fig. 1) and Sec. 4.1
 * (stencil as banded matrix products, halo of width r).
 */
mms_status mms_stencil_apply(int shape, int radius, const float *coeffs, const float *in,
                             float *out, int64_t nx, int64_t ny, int64_t nz, void *stream);

/* Full description of a sweep: shape, radius, sizes, pitches, path and an
 * optional tile-configuration index (variant; -1 = library choice, see
 * mms_num_variants). */
typedef struct {
    int32_t shape;
    int32_t radius;
    const float *coeffs;   /* host */
    int64_t nx, ny, nz;
    int64_t in_pitch_y, in_pitch_z;    /* elements, 0 = dense */
    int64_t out_pitch_y, out_pitch_z;  /* elements, 0 = dense */
    int32_t path;          /* mms_path */
    int32_t variant;       /* -1 = library choice */
} mms_stencil_desc;

/*
 * The sweep of mms_stencil_apply with explicit pitches, path and tile
 * variant.  The TMA-staged paths need in_pitch_y*4 and in_pitch_z*4 to be
 * multiples of 16 bytes and `in` 16-byte aligned; with MMS_PATH_AUTO an
 * input that breaks this runs on MMS_PATH_NAIVE, with a forced TMA path it
 * returns MMS_E_ALIGN.  Tensor-core paths support the box and the star of
 * radius 1..4.  The star's variants come in two forms.  The first half
 * (the library's choice) sweep it in one pass: the in-plane x/y part as
 * banded tensor-core products, the 2r z terms as FP32 multiply-adds on the
 * centre column of each staged plane, summed in the same kernel.  The
 * second half run two passes: the x/y part on the tensor cores into a
 * temporary grid of nx*ny*nz floats taken from the device's stream-ordered
 * memory pool (cudaMallocAsync on `stream`, freed on it after use), then
 * the z part on the CUDA cores.
 * Defined by: paper Sec. 1, Sec. 4.1 (banded products), Sec. 4.3 (box as
 * 2r+1 shifted 1D stencils per plane).
 */
mms_status mms_stencil_apply_ex(const mms_stencil_desc *desc, const float *in, float *out,
                                void *stream);

/*
 * The sweep of mms_stencil_apply_ex on grids in HOST memory: host_in and
 * host_out are host pointers with the layouts and pitches of the
 * descriptor (input pitches multiples of 4 floats).  The library streams
 * z-slabs of the input (each with its 2r halo planes; a slab of a padded
 * grid is one contiguous range) to the device, sweeps them on `stream` and
 * copies the results back, pipelined over two device slab buffers taken
 * from the device's stream-ordered memory pool and two copy streams of its
 * own, so slab k+1 is copied in while slab k is swept and slab k-1 copied
 * out.  Asynchronous: when the work queued on `stream` has finished,
 * host_out holds the result (host_in must stay unchanged until then).
 * Pinned (page-locked) host memory gives asynchronous, overlapped copies;
 * pageable memory works but its copies are staged and serialised.  Errors
 * as mms_stencil_apply_ex.
 * Defined by: the sweep above (paper Sec. 1, Sec. 4.1); the slab pipeline
 * is the GB300 analogue of the paper's streaming of planes (Sec. 4.4, 4.5).
 */
mms_status mms_stencil_apply_host(const mms_stencil_desc *desc, const float *host_in, float *host_out,
                                  void *stream);

/* The path MMS_PATH_AUTO takes for (shape, radius) on an input that does
 * (tma_aligned = 1) or does not (0) meet the TMA alignment rule above;
 * -1 for an invalid shape or radius.  AUTO takes the tensor cores (BF16x3,
 * FP32-level accuracy) where a tuned BF16x3 variant exists for (shape,
 * radius): registered with mms_set_variant, or in the library's built-in
 * table for the current device.  The built-in table is the autotuner's
 * measurements compiled into the library: on a device whose name is that of
 * the GPU the table was tuned on, it gives every (shape, radius, path) its
 * measured best variant, and it holds a BF16x3 row only where that path beat
 * the CUDA cores.  Elsewhere AUTO takes the TMA CUDA-core path (the naive
 * path for unaligned input).  Host only; the first call on a device reads
 * the device's name (cudaGetDeviceProperties). */
int32_t mms_auto_path(int shape, int radius, int tma_aligned);

/* Number of tile variants of (shape, radius, path); variant indices run
 * 0..n-1.  Returns 0 for an unsupported combination.  Host only. */
int32_t mms_num_variants(int shape, int radius, int path);

/* Library choice of variant for (shape, radius, path, nx, ny, nz): the one
 * registered by mms_set_variant, else the built-in table's row for the
 * current device (see mms_auto_path), else variant 0; -1 for an unsupported
 * combination.  The choice does not depend on the sizes at present (they are
 * in the signature so that a size-dependent table needs no ABI change).
 * Host only. */
int32_t mms_default_variant(int shape, int radius, int path, int64_t nx, int64_t ny, int64_t nz);

/* Record a tuned variant for (shape, radius, path); used by MMS_PATH_AUTO
 * and variant -1 from then on in this process, in place of the built-in
 * table.  variant -1 clears it: (shape, radius, path) then has no tuned
 * variant (variant 0; AUTO keeps a cleared BF16x3 path off), the built-in
 * row included. */
mms_status mms_set_variant(int shape, int radius, int path, int32_t variant);

/* Largest interior (nx*ny*nz points) of mms_stencil_apply_noalloc: its
 * temporary grid is a fixed device array of this many floats (32 MiB). */
#define MMS_NOALLOC_MAX_POINTS 8388608

/*
 * The star sweep on tensor cores (MMS_PATH_TF32, MMS_PATH_3XTF32 or
 * MMS_PATH_BF16X3; MMS_PATH_AUTO means MMS_PATH_BF16X3) without any device
 * allocation.  The paper has no counterpart: it is for callers that cannot
 * call cudaMalloc or a stream-ordered allocator (a host whose device memory
 * is all reserved for its own allocator, a plugin with a fixed footprint).
 * It runs the star's two-pass form: where mms_stencil_apply_ex's two-pass
 * variants take the temporary grid of nx*ny*nz floats from the device's
 * memory pool, this entry point uses a file-scope device array of
 * MMS_NOALLOC_MAX_POINTS floats, which every GPU that loads the library
 * holds until the process exits.  (The single-pass variants of
 * mms_stencil_apply_ex need no temporary grid at all.)  desc->variant picks
 * the tile (-1 = the library's choice), always in the two-pass form.
 * Arguments, layouts and results are those of mms_stencil_apply_ex with
 * shape MMS_STAR; the caller still passes the input and output.
 * Set-up: every call looks the array's device address up for the current
 * device (cudaGetSymbolAddress); the first such lookup on a device loads
 * the library's module there, so make the first call on each device
 * outside any stream capture.
 * Errors: MMS_E_ARG for nx*ny*nz above MMS_NOALLOC_MAX_POINTS, a path that
 * is not an mms_path value or a variant beyond the two-pass ones (and the
 * checks of mms_stencil_apply_ex); MMS_E_UNSUPPORTED for the box shape or
 * a CUDA-core or naive path; MMS_E_ALIGN as for the forced TMA paths.
 * Sharing: every call on a device uses the same array and leaves its
 * contents behind; nothing in it needs to start at zero (each call writes
 * the part it reads).  Calls whose work overlaps on the GPU (other streams,
 * other host threads) race on the array: serialise them, e.g. on one stream.
 */
mms_status mms_stencil_apply_noalloc(const mms_stencil_desc *desc, const float *in, float *out,
                                     void *stream);

/*
 * FP64 sweep (the paper's motivation compares GPU stencil libraries in FP64,
 * Sec. 3.2): the definition of mms_stencil_apply_ex in double precision on
 * the CUDA cores.  desc gives shape, radius, sizes and pitches (in doubles;
 * 0 = dense); desc->coeffs is not read -- the weights come in `coeffs`
 * (host doubles, layout as for mms_stencil_apply); desc->path must be
 * MMS_PATH_AUTO or MMS_PATH_CUDA_CORE and desc->variant is ignored.
 * in/out: device doubles, 8-byte aligned, not overlapping.  Bound by
 * GB300's FP64 pipe (about 2 FMAs per clock per SM): a star of radius r
 * costs 6r + 1 FMAs per point (its three centre weights folded into one),
 * a box (2r+1)^3.  Errors as for mms_stencil_apply_ex.
 */
mms_status mms_stencil_apply_f64(const mms_stencil_desc *desc, const double *coeffs, const double *in,
                                 double *out, void *stream);

/* ------------------------------------------------------- acoustic wave */

/*
 * Geometry of the damped acoustic wave step used for reverse time migration
 * (paper Sec. 2.1 names RTM with radius-4 stencils; Sec. 5.6 runs it).  The
 * paper prints no discretisation; the step is
 *     a^{n+1} = G*( (2 + m*L) a^n - G*a^{n-1} + s^n )
 * with L the star stencil of `radius` (unscaled weights), m = v^2 dt^2/h^2,
 * G = g(x) g(y) g(z) the Cerjan sponge g(d) = exp(-(a (w-d))^2) for the
 * cell at distance d < w from the nearest face (1 otherwise), and s^n the
 * source value at one point per shot.  Fields are padded by `radius` with a
 * zero halo that the library never writes; shots are stacked at
 * `shot_stride` elements.
 */
typedef struct {
    int64_t nx, ny, nz;        /* interior */
    int32_t radius;            /* 1..4 */
    int32_t nshots;            /* 1..64 */
    int64_t pitch_y, pitch_z;  /* padded field pitches (elements), 0 = dense */
    int64_t shot_stride;       /* elements between shots, 0 = pitch_z*(nz+2r) */
    int32_t sponge_width;      /* w >= 0 (0 = no sponge) */
    float sponge_a;            /* a */
    int32_t rec_z;             /* receiver plane (interior z), -1 = no records */
    const int32_t *src_xyz;    /* host, 3*nshots interior (x,y,z); x < 0 = no source */
    int64_t grad_shot_stride;  /* mms_wave_adjoint's gradient: 0 = one nz*ny*nx slice that all
                                  shots add to; >= nz*ny*nx = shot s adds to its own slice at
                                  grad_m + s*grad_shot_stride (no atomics; sum the slices with
                                  mms_sum_f64) */
} mms_wave_desc;

/*
 * Aliasing rules of the wave entry points, checked before anything is
 * queued (MMS_E_ARG, nothing written, otherwise): a buffer a call writes --
 * the new state, lam^n, rec / rec_all, ckpt, grad_m, lap_out -- overlaps
 * neither m nor any other buffer of the call, except where an entry point
 * allows an in-place update by name (p_next = p_prev).  Extents: a field is
 * nshots*shot_stride floats, m one padded field, a record nshots*ny*nx
 * floats per step, a checkpoint 2 fields, grad_m nz*ny*nx doubles (or
 * (nshots-1)*grad_shot_stride + nz*ny*nx with per-shot slices).
 */

/*
 * One forward step for all shots.
 * coeffs: host 3*(2r+1) star weights; m: device padded field (one, shared by
 * all shots; its halo is never read); p_cur: device a^n (nshots stacked);
 * p_prev: device, in a^{n-1}, out a^{n+1} (in place); src_amp: device,
 * nshots floats s^n; rec: device nshots*ny*nx floats receiving R a^{n+1}
 * (NULL = none).  Receivers are the plane z = rec_z.
 */
mms_status mms_wave_step(const mms_wave_desc *desc, const float *coeffs, const float *m,
                         const float *p_cur, float *p_prev, const float *src_amp, float *rec,
                         void *stream);

/*
 * The step of mms_wave_step with a^{n+1} written to p_next instead of over
 * a^{n-1}: p_prev is read only.  p_next may equal p_prev (then this is
 * mms_wave_step); otherwise it must overlap neither p_cur nor p_prev, and
 * its halo is left as it is (the caller keeps it zero).  Checkpoint
 * recomputation uses it to lay a segment's states out without copies.
 * Defined by: the step above (paper Sec. 2.1, Sec. 5.6 for the RTM setting).
 */
mms_status mms_wave_step_to(const mms_wave_desc *desc, const float *coeffs, const float *m,
                            const float *p_cur, const float *p_prev, float *p_next,
                            const float *src_amp, float *rec, void *stream);

/* Flags of mms_wave_forward. */
#define MMS_WAVE_GRAPH 1u  /* capture the step sequence once into a CUDA graph and replay it */

/*
 * nsteps forward steps from the states in p0 (a^{n-1}) and p1 (a^n); on
 * return p0/p1 hold the last two states (p1 = newest when nsteps is even,
 * p0 when odd: the buffers alternate).  amps: device nsteps*nshots source
 * values; rec_all: device nsteps*nshots*ny*nx (NULL = none), row n = R a^{n+1}.
 * ckpt: device buffer of (nsteps/ckpt_every) checkpoints, each 2 stacked
 * shot sets (a^{k}, a^{k-1} at k = j*ckpt_every, j = 0..), NULL = none.
 */
mms_status mms_wave_forward(const mms_wave_desc *desc, const float *coeffs, const float *m,
                            const float *amps, int32_t nsteps, float *p0, float *p1,
                            float *rec_all, float *ckpt, int32_t ckpt_every, uint32_t flags,
                            void *stream);

/*
 * One step of the discrete adjoint of mms_wave_step for all shots:
 *     lam^n = R^T r^n + (2 + L m) G lam^{n+1} - G^2 lam^{n+2}
 *     grad_m += sum_shots G lam^{n+1} (L a^n)          (FP64)
 * lam_cur: device lam^{n+1} (padded, zero halo); lam_prev: device, in
 * lam^{n+2}, out lam^n; resid: device nshots*ny*nx r^n on the receiver plane
 * (NULL = none); a_n: device forward state a^n (NULL = no gradient term);
 * grad_m: device nz*ny*nx doubles (dense), accumulated: with
 * desc->grad_shot_stride = 0 every shot adds to it (FP64 atomics); with a
 * stride, shot s adds to grad_m + s*stride only (plain read-modify-write),
 * nshots slices in all.  m must be padded (its halo values are multiplied by
 * the zero halo of lam).
 */
mms_status mms_wave_adjoint(const mms_wave_desc *desc, const float *coeffs, const float *m,
                            const float *lam_cur, float *lam_prev, const float *resid,
                            const float *a_n, double *grad_m, void *stream);

/*
 * mms_wave_step_to that also writes L a^n -- the star of `coeffs` applied
 * to p_cur, the term the step itself computes -- into lap_out at every
 * interior point (same geometry as the fields; its halo is left as it is).
 * The gradient's recompute passes it to mms_wave_adjoint_lap, which then
 * needs neither a^n's planes nor a second stencil.  lap_out: device, 16-byte
 * aligned, overlapping none of the fields (MMS_E_ARG otherwise).
 * Plumbing of the gradient path (the paper is silent on the adjoint).
 */
mms_status mms_wave_step_lap(const mms_wave_desc *desc, const float *coeffs, const float *m,
                             const float *p_cur, const float *p_prev, float *p_next, float *lap_out,
                             const float *src_amp, float *rec, void *stream);

/*
 * mms_wave_adjoint with the gradient term read from lap_a = L a^n (as
 * written by mms_wave_step_lap; interior points read) instead of being
 * computed from a^n: same lam^n, same gradient up to the summation order of
 * L a^n.  lap_a NULL = no gradient term.
 */
mms_status mms_wave_adjoint_lap(const mms_wave_desc *desc, const float *coeffs, const float *m,
                                const float *lam_cur, float *lam_prev, const float *resid,
                                const float *lap_a, double *grad_m, void *stream);

/*
 * The adjoint step of mms_wave_adjoint_lap in the scaled variable
 * mu = m G lam (pointwise), which the gradient path may carry instead of lam:
 *     mu^n = G (2 mu^{n+1} + m L mu^{n+1} - G mu^{n+2} + m R^T r^n)
 *     grad_m += sum_shots mu^{n+1} (L a^n)                 (FP64)
 * (lam's update multiplied by m G at the output point).  It has the forward
 * step's form -- the stencil applied to the state itself -- and runs on the
 * forward step's kernel.  Its gradient sum is m times mms_wave_adjoint_lap's
 * (mu^{n+1} = m G lam^{n+1}, and m does not change with n): divide it by m
 * once, after the last step, with mms_grad_divide_m.  mu_cur: device
 * mu^{n+1}; mu_prev: device, in mu^{n+2}, out mu^n; resid, lap_a (= L a^n,
 * as written by mms_wave_step_lap), grad_m and the per-shot gradient slices
 * as in mms_wave_adjoint_lap; lap_a NULL = no gradient term.  Needs m > 0
 * at every interior point (v != 0): mu loses lam where m = 0.  Aliasing and
 * alignment errors as mms_wave_adjoint_lap.  The paper is silent on the
 * adjoint; this is the gradient path's own formulation.
 */
mms_status mms_wave_adjoint_scaled(const mms_wave_desc *desc, const float *coeffs, const float *m,
                                   const float *mu_cur, float *mu_prev, const float *resid,
                                   const float *lap_a, double *grad_m, void *stream);

/*
 * grad_m[(z*ny + y)*nx + x] /= m at interior point (x, y, z), in FP64, for the
 * nz*ny*nx doubles of grad_m (device, dense); m: device padded field of the
 * descriptor's geometry.  Turns mms_wave_adjoint_scaled's gradient sum into
 * dJ/dm.  MMS_E_ARG for null pointers or grad_m overlapping m.
 */
mms_status mms_grad_divide_m(const mms_wave_desc *desc, const float *m, double *grad_m, void *stream);

/* m = v^2 dt^2 / h^2 into a padded field (halo set to 0); v dense nz*ny*nx.
 * MMS_E_ARG for null pointers, dt or h not positive, or m overlapping v. */
mms_status mms_model_from_velocity(const mms_wave_desc *desc, const float *v, float *m,
                                   float dt, float h, void *stream);

/* grad_v = grad_m * 2 v dt^2 / h^2 (chain rule of m = v^2 dt^2/h^2), n values.
 * grad_v may be grad_m itself (element-wise); MMS_E_ARG when it overlaps v,
 * or grad_m without being it. */
mms_status mms_grad_to_velocity(const double *grad_m, const float *v, double *grad_v, int64_t n,
                                float dt, float h, void *stream);

/* result[0] = sum_i a[i]*b[i] in FP64 over n floats (device in, device out).
 * MMS_E_ARG when result overlaps a or b. */
mms_status mms_dot_f64(const float *a, const float *b, int64_t n, double *result, void *stream);

/* out[i] = sum_{s < nslices} slices[s*stride + i], i < n, in FP64 (device in,
 * device out): the per-shot gradient slices of mms_wave_adjoint summed.
 * stride >= n; out may be slices itself (the first slice) but no other
 * slice.  Plumbing of the gradient path (paper silent on the adjoint). */
mms_status mms_sum_f64(const double *slices, int32_t nslices, int64_t stride, int64_t n, double *out,
                       void *stream);

/* ------------------------------------------------- anisotropic media */

/*
 * VTI medium (paper Sec. 2.1): from dense interior arrays vp, eps, delta
 * (nz*ny*nx floats each, device) writes two padded fields in the geometry of
 * `desc` (halo 0): mv = vp^2 dt^2/h^2 sqrt(1 + 2 delta) and
 * rho = (1 + 2 eps) / sqrt(1 + 2 delta).  Requires 1 + 2 delta > 0.
 * MMS_E_ARG for null pointers or dt, h not positive.
 */
mms_status mms_vti_model(const mms_wave_desc *desc, const float *vp, const float *eps, const float *delta,
                         float *mv, float *rho, float dt, float h, void *stream);

/*
 * One step of the VTI system of the paper's Sec. 2.1, as printed there
 * (sigma_H, sigma_V the horizontal and vertical stresses), for all shots:
 *     sH^{n+1} = G*( 2 sH^n - G*sH^{n-1} + mv*(rho*Lh sH^n + Lz sV^n) + s^n )
 *     sV^{n+1} = G*( 2 sV^n - G*sV^{n-1} + mv*(Lh sV^n + rho*Lz sH^n) + s^n )
 * i.e. mh = mv*rho = m(1 + 2 eps) and mv = m sqrt(1 + 2 delta) multiply the
 * printed terms; Lh = the x and y rows of the star weights `coeffs` (host,
 * 3*(2r+1), unscaled), Lz = the z row; G, the source (added to both
 * stresses), the zero halo, shots and pitches as for mms_wave_step.
 * mv, rho: padded medium fields of mms_vti_model (one for all shots).
 * sh_cur, sv_cur, sh_prev, sv_prev: device, read; sh_next, sv_next: device,
 * written (interior only), each either the matching *_prev field (in place)
 * or a field overlapping none of the others.  rec: device nshots*ny*nx
 * receiving sH^{n+1} on the plane rec_z (NULL = none).  All fields 16-byte
 * aligned (MMS_E_ALIGN otherwise); MMS_E_ARG for overlaps or null pointers.
 */
mms_status mms_vti_step(const mms_wave_desc *desc, const float *coeffs, const float *mv, const float *rho,
                        const float *sh_cur, const float *sv_cur, const float *sh_prev, const float *sv_prev,
                        float *sh_next, float *sv_next, const float *src_amp, float *rec, void *stream);

/*
 * TTI medium (paper Sec. 2.1): from dense interior arrays (nz*ny*nx floats
 * each, device) vp, vs, eps, delta, alpha, theta (tilt), phi (azimuth),
 * writes `med`, 8 dense interior fields one after another:
 *     [a, b, c, d, alpha, nx, ny, nz]
 * a = vpx^2 s = vp^2 (1 + 2 eps) s, b = vpz^2 s = vp^2 s,
 * c = vpn^2 s = vp^2 (1 + 2 delta) s, d = vsz^2 s = vs^2 s (s = dt^2/h^2),
 * and the tilt axis n = (sin th cos ph, sin th sin ph, cos th).  The paper
 * names vpx, vpz, vpn, vsz and alpha without defining them; these are the
 * usual Thomsen-parameter readings.  MMS_E_ARG for null pointers or dt, h
 * not positive.
 */
mms_status mms_tti_model(const mms_wave_desc *desc, const float *vp, const float *vs, const float *eps,
                         const float *delta, const float *alpha, const float *theta, const float *phi,
                         float *med, float dt, float h, void *stream);

/*
 * One step of the TTI system of the paper's Sec. 2.1 for all shots:
 *     p^{n+1} = G*( 2 p^n - G*p^{n-1} + a H2p + alpha b H1q + d (H1p - alpha H1q) + s^n )
 *     q^{n+1} = G*( 2 q^n - G*q^{n-1} + c/alpha H2p + b H1q - d (H2p/alpha - H2q) + s^n )
 * with H1 f = nx^2 f_xx + ny^2 f_yy + nz^2 f_zz + 2 nx ny f_xy + 2 ny nz f_yz
 * + 2 nx nz f_xz and H2 f = f_xx + f_yy + f_zz - H1 f.  Axis derivatives use
 * the second-derivative weights w2 (host, 2r+1 floats, offsets -r..r); a
 * mixed derivative composes two first-derivative rows w1 (host, 2r+1 floats,
 * offsets -r..r) on the zero-padded field (paper Sec. 4.7).  med: the 8
 * dense fields of mms_tti_model.  Fields, shots, G, source (added to p and
 * q), receivers (p^{n+1} on rec_z) and overlap rules as for mms_vti_step.
 * work: device scratch of 4*nshots*nx*ny*nz floats, 16-byte aligned,
 * overlapping no field, owned by the caller (the call allocates nothing).
 * Launches on `stream`: with nx a multiple of 4, two (the derivative pass of
 * p, then the pass of q with the coupling and the update fused in); other
 * sizes three (the two passes and a pointwise combine).
 */
mms_status mms_tti_step(const mms_wave_desc *desc, const float *w2, const float *w1, const float *med,
                        const float *p_cur, const float *q_cur, const float *p_prev, const float *q_prev,
                        float *p_next, float *q_next, float *work, const float *src_amp, float *rec,
                        void *stream);

/* Tile variants of the anisotropic steps (kind 0 = VTI): their count, and
 * the one used by later calls of this process (MMS_E_ARG out of range). */
int32_t mms_aniso_num_variants(int32_t kind);
mms_status mms_aniso_set_variant(int32_t kind, int32_t variant);

/* ------------------------------------------------------------ status */

/* Thread-local message of the last non-OK status of this thread. */
const char *mms_last_error(void);

/* Synchronises `stream`, reads and clears the device error word of the
 * current device: MMS_OK, MMS_E_TIMEOUT or MMS_E_DEVICE (or MMS_E_CUDA if
 * the synchronisation itself failed). */
mms_status mms_check_device(void *stream);

/*
 * Failure-detection self-test (no counterpart in the paper): queues on
 * `stream` a one-block kernel whose bounded wait on an mbarrier phase that
 * nothing completes runs out after limit_us microseconds (1..2000000).  Like
 * every bounded wait of the library's kernels, it then sets the timeout bit
 * of the device error word and returns, so the next mms_check_device returns
 * MMS_E_TIMEOUT and the context stays usable.  MMS_E_ARG for a limit out of
 * range.
 */
mms_status mms_selftest_timeout(uint32_t limit_us, void *stream);

/*
 * The pipeline constants of the tensor-core sweep of (shape, radius, path)
 * in this build, for checking its schedule on the host (no device is
 * touched; the producer stages planes into a ring, one issuer runs every
 * output's products in order, workers convert planes and drain outputs).
 * cfg receives up to ncfg of, in order: mixed (1 if the two workers of a
 * lane quarter each convert the planes and drain the outputs of one
 * parity), look (planes a mixed worker converts past the last plane its
 * next output reads), a_ring (planes the tensor-memory operand ring holds),
 * staging (planes the shared-memory staging ring holds), accumulators,
 * reach (planes an output reads, or waits for, past its first), z_halo
 * (halo planes a tile stages on each side in z), two_ctas (1 if two CTAs
 * share an SM), drainers (warps per lane quarter that drain outputs).
 * Returns the number of constants (9), or -1 for a shape, radius or path
 * without a tensor-core sweep, or a null cfg with ncfg > 0.
 */
int32_t mms_tc_pipeline_config(int32_t shape, int32_t radius, int32_t path, int32_t *cfg, int32_t ncfg);

/* Library version string. */
const char *mms_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MMS_H */
