// readout.cuh -- the read-outs of the Gram (device code shared by every
// kernel that produces PLV / iPLV / ciPLV, so the fused epilogues and the
// stand-alone metrics kernel give identical bits).
#pragma once

#include <cuda_runtime.h>

namespace plv {

// Denominator of Eq. 14, d = 1 - (Re C)^2, formed as (1 - r)(1 + r) in
// FP32, which does not cancel: for |r| >= 1/2 the factor 1 - |r| is exact
// (Sterbenz's lemma: 1 and |r| are within a factor of two) and the other
// factor lies in [3/2, 2) with at most half an ulp of rounding; below 1/2
// both factors lie in (1/2, 3/2).  So d carries about one ulp of relative
// rounding in every range, far below the effect of the input's own error
// (2 |r| dr).  Forming it in FP64 changes d by at most that ulp.
__device__ __forceinline__ float ciplv_den(float r) {
    return (1.0f - r) * (1.0f + r);
}

// PLV = |C| (Eq. 7), iPLV = |Im C| (Eq. 13, in absolute value) and
// ciPLV = Im C / sqrt((1 - Re C)(1 + Re C)) (Eq. 14) of one off-diagonal
// Gram entry C = re + i im already scaled by 1/T; ciPLV = 0 where the
// denominator is not positive.
__device__ __forceinline__ void readout(float re, float im, float &plv,
                                        float &iplv, float &ciplv) {
    plv = sqrtf(fmaf(re, re, im * im));
    iplv = fabsf(im);
    const float d = ciplv_den(re);
    ciplv = d > 0.0f ? im / sqrtf(d) : 0.0f;
}

}  // namespace plv
