// sweep_star.cu -- the FP32 CUDA-core star sweeps (kernel in sweep_cc.cuh,
// design notes in sweep_cc.cu): the tile variants of the star and their
// dispatch, in a translation unit of their own so that the two shapes
// compile in parallel.
#include "sweep_cc.cuh"

namespace mms {
namespace {

using sweep::Variant;
using sweep::launch_tiled;

// Star tile variants (TX, TY, PY, stages, TZ, rotated queue, one waiter).
constexpr Variant kStarVariants[] = {
    {64, 16, 2, 4, 128, false},       {64, 32, 4, 3, 128, false},       {128, 32, 2, 3, 64, false},
    {64, 16, 2, 3, 128, false, true}, {64, 16, 2, 4, 128, true},        {64, 32, 2, 4, 128, false, true},
    {128, 32, 2, 3, 64, true},        {64, 16, 2, 4, 128, true, true},  {128, 32, 2, 3, 64, true, true},
    {64, 32, 4, 3, 128, false, true}, {64, 16, 2, 4, 128, false, true}, {128, 16, 2, 4, 128, false, true},
    // 256-plane z chunks: half the z-halo re-reads of the 128-plane ones
    {64, 16, 2, 4, 256, false, true}, {64, 16, 2, 3, 256, false, true},
};
constexpr int kNumStar = sizeof(kStarVariants) / sizeof(Variant);

template <int R>
cudaError_t dispatch_star(const Sweep &sw, const CUtensorMap &tmap, const StarCoef &cf, int v)
{
    MMS_SWEEP_DISPATCH(kStarVariants, R, false, StarCoef, sw, tmap, cf, v)
}

}  // namespace

int star_cc_variants() { return kNumStar; }

void star_cc_box(int r, int v, int *bx, int *by)
{
    const Variant &t = kStarVariants[v];
    *bx = (t.tx + 2 * r + 3) & ~3;
    *by = t.ty + 2 * r;
}

cudaError_t launch_star_cc(const Sweep &s, const CUtensorMap &tmap, int v)
{
    StarCoef cf{};
    const int w = 2 * s.r + 1;
    for (int i = 0; i < 3 * w; ++i) cf.c[i] = s.coeffs[i];
    switch (s.r) {
        case 1: return dispatch_star<1>(s, tmap, cf, v);
        case 2: return dispatch_star<2>(s, tmap, cf, v);
        case 3: return dispatch_star<3>(s, tmap, cf, v);
        case 4: return dispatch_star<4>(s, tmap, cf, v);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mms
