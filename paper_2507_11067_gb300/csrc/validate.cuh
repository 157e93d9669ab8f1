// validate.cuh -- host-side checks of caller-given geometry, shared by the ABI
// entry points (abi.cu, noalloc.cu).
#pragma once

#include <stdint.h>

namespace mms {

// Largest span (elements) a caller-given pitch or stride may describe: far
// beyond any device memory, and small enough that no extent computed from
// sizes below 2^30 and such pitches overflows 64 bits.
constexpr int64_t kMaxSpan = int64_t(1) << 46;

// The pitches of a (Z, Y, X) grid (Y, Z >= 1) from the caller's values, 0
// meaning dense (py = X, pz = Y*py); false unless both are positive with
// Y*py and Z*pz at most kMaxSpan.  Each default is formed only after the
// pitch it multiplies has been bounded, so nothing here overflows.
inline bool resolve_pitches(int64_t X, int64_t Y, int64_t Z, int64_t py_in, int64_t pz_in, int64_t *py,
                            int64_t *pz)
{
    *py = py_in ? py_in : X;
    if (*py <= 0 || *py > kMaxSpan / Y) return false;
    *pz = pz_in ? pz_in : Y * *py;
    return *pz > 0 && *pz <= kMaxSpan / Z;
}

}  // namespace mms
