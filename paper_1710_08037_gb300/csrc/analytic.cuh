// analytic.cuh -- the K1 tasks (what the FFT engine of fft.cuh reads and
// writes for the forward phasors and for the backward recompute) and the
// store of a unit phasor in the Gram's operand layout.  Shared by the K1
// translation units; the launchers are compiled once per (input type, task)
// in k_fwd.cu.
//
// The real part of the discrete analytic signal equals the input exactly
// (the analytic mask satisfies h[k] + h[-k] = 2), so z = x + i H{x} with H{x}
// from the engine and x re-read at the end (an L2 hit).
#pragma once

#include "fft.cuh"

namespace plv {

// Task kinds of K1: the forward phasors in each operand precision, and the
// backward recompute (FP32 phasors and reciprocal amplitudes).
enum K1Kind { kK1Fp32 = PLV_PREC_FP32, kK1Bf16 = PLV_PREC_BF16X3, kK1Fp16 = PLV_PREC_FP16X3,
              kK1Prep = 3 };

// Arguments of one K1 launch over `rows` rows of x (row r = e * N + n).
struct K1Args {
    const void *x;
    int64_t ldx;
    void *P;        // phasors (operand layout of the kind)
    float *rinv;    // kK1Prep only: [rows][ld] reciprocal amplitudes
    int N, T, log2T;
    int64_t ld;     // padded row length
    int64_t rows;
};

// Launchers, defined in k_fwd.cu and instantiated there once per
// (Tin, KIND): the direct power-of-two engine, the any-length engine, and the
// grouped any-length launch over many problems (forward kinds only).
template <typename Tin, int KIND>
cudaError_t k1_pow2(const Handle *h, cudaStream_t s, const K1Args &a);
template <typename Tin, int KIND>
cudaError_t k1_conv(const Handle *h, cudaStream_t s, const K1Args &a, const ConvPlan &plan);
template <typename Tin, int KIND>
cudaError_t k1_conv_group(const Handle *h, cudaStream_t s, const K1Group &g);

#define PLV_K1_EXTERN(TIN, KIND)                                                              \
    extern template cudaError_t k1_pow2<TIN, KIND>(const Handle *, cudaStream_t,              \
                                                   const K1Args &);                           \
    extern template cudaError_t k1_conv<TIN, KIND>(const Handle *, cudaStream_t,              \
                                                   const K1Args &, const ConvPlan &);         \
    extern template cudaError_t k1_conv_group<TIN, KIND>(const Handle *, cudaStream_t,        \
                                                         const K1Group &);
PLV_K1_EXTERN(float, kK1Fp32)
PLV_K1_EXTERN(double, kK1Fp32)
PLV_K1_EXTERN(float, kK1Bf16)
PLV_K1_EXTERN(double, kK1Bf16)
PLV_K1_EXTERN(float, kK1Fp16)
PLV_K1_EXTERN(double, kK1Fp16)
PLV_K1_EXTERN(float, kK1Prep)
PLV_K1_EXTERN(double, kK1Prep)
#undef PLV_K1_EXTERN

namespace {

using namespace fft;

template <typename Tin>
__device__ __forceinline__ float ldx_f(const Tin *p) {
    return (float)__ldg(p);
}

// Where row r (= e * N + n) of the operand layout starts: the FP32 planar
// row (float index), or, for the tiled split layout, the row's element base
// within its row block plus its swizzle key.
template <int PREC>
struct RowAddr {
    int64_t base;
    int sw;
};
template <int PREC>
__device__ __forceinline__ RowAddr<PREC> row_addr(int64_t r, int N, int64_t ld) {
    RowAddr<PREC> a;
    if constexpr (PREC == PLV_PREC_FP32) {
        a.base = r * 2 * ld;
        a.sw = 0;
    } else {
        const int64_t e = r / N, n = r - e * N;
        const int64_t rb = n >> 7, rr = n & 127;
        a.base = (e * row_blocks(N) + rb) * (ld / kTileK) * kBlockElems + rr * kTileK;
        a.sw = (int)((rr >> 1) & 3);
    }
    return a;
}

// Store one unit phasor at sample m of a row: FP32 planar, or the tiled split
// layout (common.cuh) with each component split as hi = RN(p), lo = RN(p - hi).
template <int PREC>
__device__ __forceinline__ void store_phasor(void *P, const RowAddr<PREC> &ra, int64_t ld,
                                             int m, float2 p) {
    if constexpr (PREC == PLV_PREC_FP32) {
        float *o = (float *)P + ra.base + m;
        o[0] = p.x;
        o[ld] = p.y;
    } else {
        const int k = m & 31;
        const int64_t off = ra.base + (int64_t)(m >> 5) * kBlockElems +
                            ((((k >> 3) ^ ra.sw) << 3) | (k & 7));
        constexpr int64_t ps = kTileRows * kTileK;  // plane stride in a block
        if constexpr (PREC == PLV_PREC_FP16X3) {
            __half *o = (__half *)P + off;
            const __half rh = __float2half_rn(p.x);
            const __half ih = __float2half_rn(p.y);
            o[0] = rh;
            o[ps] = __float2half_rn(p.x - __half2float(rh));
            o[2 * ps] = ih;
            o[3 * ps] = __float2half_rn(p.y - __half2float(ih));
        } else {
            __nv_bfloat16 *o = (__nv_bfloat16 *)P + off;
            const __nv_bfloat16 rh = __float2bfloat16_rn(p.x);
            const __nv_bfloat16 ih = __float2bfloat16_rn(p.y);
            o[0] = rh;
            o[ps] = __float2bfloat16_rn(p.x - __bfloat162float(rh));
            o[2 * ps] = ih;
            o[3 * ps] = __float2bfloat16_rn(p.y - __bfloat162float(ih));
        }
    }
}

// Forward task: rows of x in, phasors P = z/|z| in the operand layout out
// (z = x + i H{x}; |z|^2 below the rounding floor counts as |z| = 0).
template <typename Tin, int PREC>
struct FwdTask {
    const Tin *x;
    int64_t ldx;
    void *P;
    int N;
    int64_t ld;
    struct Rows {
        const Tin *x0, *x1;  // nullptr for a row past the end
        RowAddr<PREC> a0, a1;
    };
    __device__ Rows rows(int64_t r0, bool v0, int64_t r1, bool v1) const {
        Rows rs;
        rs.x0 = v0 ? x + r0 * ldx : nullptr;
        rs.x1 = v1 ? x + r1 * ldx : nullptr;
        rs.a0 = row_addr<PREC>(v0 ? r0 : 0, N, ld);
        rs.a1 = row_addr<PREC>(v1 ? r1 : 0, N, ld);
        return rs;
    }
    __device__ float2 load(const Rows &rs, int m) const {
        return make_float2(rs.x0 ? ldx_f(rs.x0 + m) : 0.f, rs.x1 ? ldx_f(rs.x1 + m) : 0.f);
    }
    __device__ void finish(const Rows &rs, int m, float h0, float h1, float floor2) const {
        if (rs.x0) store_phasor<PREC>(P, rs.a0, ld, m, unit_phasor(ldx_f(rs.x0 + m), h0, floor2));
        if (rs.x1) store_phasor<PREC>(P, rs.a1, ld, m, unit_phasor(ldx_f(rs.x1 + m), h1, floor2));
    }
    // padding samples T <= m < ld are zero
    __device__ void pad(const Rows &rs, int m) const {
        if (rs.x0) store_phasor<PREC>(P, rs.a0, ld, m, make_float2(0.f, 0.f));
        if (rs.x1) store_phasor<PREC>(P, rs.a1, ld, m, make_float2(0.f, 0.f));
    }
};

// Backward preparation: the same analytic signal, stored as FP32 phasors
// P[row][2][ld] and the reciprocal amplitude rinv[row][ld] = 1/|z| (0 where
// |z| counts as 0), which the gradient of Eq. 4 needs.
template <typename Tin>
struct PrepTask {
    const Tin *x;
    int64_t ldx;
    float *P;
    float *rinv;
    int64_t ld;
    struct Rows {
        const Tin *x0, *x1;
        float *p0, *p1, *q0, *q1;  // phasor rows, reciprocal-amplitude rows
    };
    __device__ Rows rows(int64_t r0, bool v0, int64_t r1, bool v1) const {
        Rows rs;
        rs.x0 = v0 ? x + r0 * ldx : nullptr;
        rs.x1 = v1 ? x + r1 * ldx : nullptr;
        rs.p0 = P + (v0 ? r0 : 0) * 2 * ld;
        rs.p1 = P + (v1 ? r1 : 0) * 2 * ld;
        rs.q0 = rinv + (v0 ? r0 : 0) * ld;
        rs.q1 = rinv + (v1 ? r1 : 0) * ld;
        return rs;
    }
    __device__ void one(const Tin *xr, float *pr, float *qr, int m, float h,
                        float floor2) const {
        float ri;
        const float2 p = unit_phasor_inv(ldx_f(xr + m), h, floor2, ri);
        pr[m] = p.x;
        pr[ld + m] = p.y;
        qr[m] = ri;
    }
    __device__ float2 load(const Rows &rs, int m) const {
        return make_float2(rs.x0 ? ldx_f(rs.x0 + m) : 0.f, rs.x1 ? ldx_f(rs.x1 + m) : 0.f);
    }
    __device__ void finish(const Rows &rs, int m, float h0, float h1, float floor2) const {
        if (rs.x0) one(rs.x0, rs.p0, rs.q0, m, h0, floor2);
        if (rs.x1) one(rs.x1, rs.p1, rs.q1, m, h1, floor2);
    }
    __device__ void pad(const Rows &rs, int m) const {
        if (rs.x0) { rs.p0[m] = 0.f; rs.p0[ld + m] = 0.f; rs.q0[m] = 0.f; }
        if (rs.x1) { rs.p1[m] = 0.f; rs.p1[ld + m] = 0.f; rs.q1[m] = 0.f; }
    }
};

}  // namespace
}  // namespace plv
