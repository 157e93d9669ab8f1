// wave.cuh -- internal interface of the fused acoustic wave kernels.
#pragma once

#include "common.cuh"

namespace mms {

constexpr int kMaxShots = 64;

// Geometry of a batched wave step, as validated by the ABI layer.
struct WaveGeo {
    int nx, ny, nz, r, nshots;
    int64_t py, pz, ss;  // padded pitches and shot stride (elements)
    int sponge_w;
    float sponge_a;
    int rec_z;
    int64_t gss;  // per-shot gradient slice stride (0 = one shared slice, atomics)
    int src[kMaxShots][3];
};

// a^{n+1} goes to p_next (== p_prev for the in-place step); with lapout,
// L a^n of every interior point goes there too (same geometry).
cudaError_t launch_wave_fwd(const WaveGeo &g, const float *coeffs, const float *m, const float *p_cur,
                            const float *p_prev, float *p_next, const float *src_amp, float *rec,
                            cudaStream_t st, float *lapout = nullptr);
// The adjoint step in mu = m g lam (the gradient path): mu^n into mu_prev
// (which held mu^{n+2}); with lap_a and grad, grad += mu^{n+1} (L a^n).
cudaError_t launch_wave_adj_scaled(const WaveGeo &g, const float *coeffs, const float *m, const float *mu_cur,
                                   float *mu_prev, const float *resid, const float *lap_a, double *grad,
                                   cudaStream_t st);
// lapin: a_n holds L a^n (interior read) instead of a^n.
cudaError_t launch_wave_adj(const WaveGeo &g, const float *coeffs, const float *m, const float *lam_cur,
                            float *lam_prev, const float *resid, const float *a_n, double *grad,
                            cudaStream_t st, bool lapin = false);
cudaError_t launch_model_from_velocity(const WaveGeo &g, const float *v, float *m, float dt, float h,
                                       cudaStream_t st);
// grad (dense nz*ny*nx FP64) divided by m at each interior point.
cudaError_t launch_grad_divide_m(const WaveGeo &g, const float *m, double *grad, cudaStream_t st);
cudaError_t launch_grad_to_velocity(const double *gm, const float *v, double *gv, int64_t n, float dt,
                                    float h, cudaStream_t st);
cudaError_t launch_dot_f64(const float *a, const float *b, int64_t n, double *res, cudaStream_t st);
cudaError_t launch_wait_selftest(unsigned long long limit_ns, cudaStream_t st);
cudaError_t launch_sum_f64(const double *slices, int nslices, int64_t stride, int64_t n, double *out,
                           cudaStream_t st);

// VTI step (aniso.cu): sigma_H, sigma_V at n+1 into hnext/vnext (which may
// be hprev/vprev); medium mv, rho padded like the fields (one, all shots).
cudaError_t launch_vti_step(const WaveGeo &g, const float *coeffs, const float *mv, const float *rho,
                            const float *hcur, const float *vcur, const float *hprev, const float *vprev,
                            float *hnext, float *vnext, const float *src_amp, float *rec, cudaStream_t st);
cudaError_t launch_vti_model(const WaveGeo &g, const float *vp, const float *eps, const float *delta, float *mv,
                             float *rho, float dt, float h, cudaStream_t st);
// TTI step (aniso.cu): derivative passes for p and q into `work` (4 *
// nshots * nx*ny*nz floats: Lap p, H1 p, Lap q, H1 q), then the combine into
// pn/qn (which may be pp/qp).  med: 8 dense interior fields.
cudaError_t launch_tti_step(const WaveGeo &g, const float *w2, const float *w1, const float *med,
                            const float *pc, const float *qc, const float *pp, const float *qp, float *pn, float *qn,
                            float *work, const float *src_amp, float *rec, cudaStream_t st);
cudaError_t launch_tti_model(int64_t n, const float *vp, const float *vs, const float *eps, const float *delta,
                             const float *alpha, const float *theta, const float *phi, float *med, float dt, float h,
                             cudaStream_t st);
int vti_num_variants();
bool vti_set_variant(int v);

// Cerjan sponge factor of cell i of n (distance d to the nearest face).
__device__ __forceinline__ float sponge(int i, int n, int w, float a)
{
    const int d = min(i, n - 1 - i);
    if (d < w) {
        const float t = a * (float)(w - d);
        return expf(-t * t);
    }
    return 1.f;
}

// Interior tile (TX x TY) of m or a^{n-1} that completes with output plane
// zo: TMA box x start rounded down to a 16-byte boundary, OFF columns in.
template <int R, int TX>
struct Interior {
    static constexpr int OFF = R % 4;                   // column of output x0 inside the box
    static constexpr int BXI = OFF == 0 ? TX : TX + 4;  // box width (16-byte multiple)
};

mms_status fail(mms_status st, const char *fmt, ...);
mms_status cuda_fail(cudaError_t e, const char *what);

}  // namespace mms
