// band_tc.cu -- tensor-core banded sweeps (tcgen05); filled in below.
#include "common.cuh"

namespace mms {

int band_tc_supported(int, int, int) { return 0; }
int band_tc_variants(int, int, int) { return 0; }
void band_tc_box(int, int, int, int, int *bx, int *by, int *bz) { *bx = *by = *bz = 0; }
cudaError_t launch_band_tc(const Sweep &, int, const CUtensorMap &, int) { return cudaErrorNotSupported; }

}  // namespace mms
