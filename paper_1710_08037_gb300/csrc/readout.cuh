// readout.cuh -- the read-outs of the Gram (device code shared by every
// kernel that produces PLV / iPLV / ciPLV, so the fused epilogues and the
// stand-alone metrics kernel give identical bits).
#pragma once

#include <cuda_runtime.h>

namespace plv {

// PLV = |C| (Eq. 7), iPLV = |Im C| (Eq. 13, in absolute value) and
// ciPLV = Im C / sqrt((1 - Re C)(1 + Re C)) (Eq. 14) of one Gram entry
// C = re + i im that has already been scaled by 1/T.  The denominator is
// formed in FP64 in the factored form, which does not cancel as |Re C| -> 1;
// where it is not positive ciPLV is 0.
__device__ __forceinline__ void readout(float re, float im, float &plv,
                                        float &iplv, float &ciplv) {
    plv = sqrtf(fmaf(re, re, im * im));
    iplv = fabsf(im);
    const double r = (double)re;
    const double d = (1.0 - r) * (1.0 + r);
    ciplv = d > 0.0 ? im / sqrtf((float)d) : 0.0f;
}

}  // namespace plv
