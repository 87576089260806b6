// readout.cuh -- the read-outs of the Gram (device code shared by every
// kernel that produces PLV / iPLV / ciPLV, so the fused epilogues and the
// stand-alone metrics kernel give identical bits).
#pragma once

#include <cuda_runtime.h>

namespace plv {

// Denominator of Eq. 14, d = 1 - (Re C)^2, formed as (1 - r)(1 + r).  Where
// the plain 1 - r^2 would cancel, |r| > 1 - 2^-6 (d < 2^-5), the factors and
// their product are taken in FP64, so d is the exactly rounded FP32 value of
// the FP32 input's true denominator.  Below that threshold the FP32 factored
// form already carries about one ulp: for |r| >= 1/2 the factor 1 - |r| is
// exact (Sterbenz's lemma) and the other lies in [3/2, 2) with at most half
// an ulp of rounding; below 1/2 both factors lie in (1/2, 3/2).  Either way
// the rounding of d is far below the effect of the Gram's own error in r
// (2 |r| dr).
constexpr float kCiplvFp64Above = 1.0f - 0x1p-6f;
__device__ __forceinline__ float ciplv_den(float r) {
    if (fabsf(r) > kCiplvFp64Above) {
        const double rd = (double)r;
        return (float)((1.0 - rd) * (1.0 + rd));
    }
    return (1.0f - r) * (1.0f + r);
}

// The square root and the division of the read-outs go through the
// special-function unit's reciprocal square root (rsqrtf, a few ulp) rather
// than IEEE sqrtf and division: the read-outs already carry the Gram's own
// error (about 1e-6 absolute), far above either rounding, and the epilogue
// spends most of its instructions here.

// |C| = sqrt(re^2 + im^2), 0 at C = 0.
__device__ __forceinline__ float plv_of(float re, float im) {
    const float r2 = fmaf(re, re, im * im);
    return r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f;
}

// Im C / sqrt(d) for d = ciplv_den(Re C), 0 where d is not positive.
__device__ __forceinline__ float ciplv_of(float re, float im) {
    const float d = ciplv_den(re);
    return d > 0.0f ? im * rsqrtf(d) : 0.0f;
}

// PLV = |C| (Eq. 7), iPLV = |Im C| (Eq. 13, in absolute value) and
// ciPLV = Im C / sqrt((1 - Re C)(1 + Re C)) (Eq. 14) of one off-diagonal
// Gram entry C = re + i im already scaled by 1/T; ciPLV = 0 where the
// denominator is not positive.
__device__ __forceinline__ void readout(float re, float im, float &plv,
                                        float &iplv, float &ciplv) {
    plv = plv_of(re, im);
    iplv = fabsf(im);
    ciplv = ciplv_of(re, im);
}

}  // namespace plv
