// readout.cuh -- the read-outs of the Gram (device code shared by every
// kernel that produces PLV / iPLV / ciPLV, so the fused epilogues and the
// stand-alone metrics kernel give identical bits).
#pragma once

#include <cuda_runtime.h>

namespace plv {

// Denominator of Eq. 14, d = 1 - (Re C)^2 = (1 - a)(1 + a), a = |Re C|,
// formed without cancellation and to the accuracy of an FP64 evaluation,
// with an error-free transformation in FP32 (no FP64 instruction, no branch):
//   u = 1 - a              exact for a >= 1/2 (Sterbenz's lemma);
//   v = RN(1 + a), e = (1 - v) + a, so v + e = 1 + a exactly (Fast2Sum);
//   p = RN(u v), pe = fma(u, v, -p), so u v = p + pe exactly;
//   d = RN(p + fma(u, e, pe))  =  u (1 + a) with two final roundings,
// within one ulp of the correctly rounded exact value -- the value that the
// factors and product taken in FP64 and rounded to FP32 give -- in the range
// where 1 - Re^2 cancels (a -> 1).  Below a = 1/2, where nothing cancels, u
// carries half an ulp.  An FP64 branch for |Re| > 1 - 2^-6 gave the same
// values but, taken or not, cost 30-53 % of the epilogue-bound Grams (K = 64
// trials, short windows) on GB300's slow FP64 pipe.
__device__ __forceinline__ float ciplv_den(float r) {
    const float a = fabsf(r);
    const float u = 1.0f - a;
    const float v = 1.0f + a;
    const float e = (1.0f - v) + a;
    const float p = u * v;
    const float pe = fmaf(u, v, -p);
    return p + fmaf(u, e, pe);
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
