// sweep_box_high.cu -- the FP32 CUDA-core box sweeps of radius 3 and 4
// (kernel in sweep_cc.cuh, design notes in sweep_cc.cu), in a translation
// unit of their own: their (2r+1)^3-term plane updates are the largest
// instantiations and compile in parallel with the rest.
#include "sweep_cc.cuh"

namespace mms {
namespace sweep {

namespace {

template <int R>
cudaError_t dispatch_box_high(const Sweep &sw, const CUtensorMap &tmap, const BoxCoef &cf, int v)
{
    MMS_SWEEP_DISPATCH(kBoxVariants, R, true, BoxCoef, sw, tmap, cf, v)
}

}  // namespace

cudaError_t launch_box_cc_high(const Sweep &s, const CUtensorMap &tmap, const BoxCoef &cf, int v)
{
    switch (s.r) {
        case 3: return dispatch_box_high<3>(s, tmap, cf, v);
        case 4: return dispatch_box_high<4>(s, tmap, cf, v);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sweep
}  // namespace mms
