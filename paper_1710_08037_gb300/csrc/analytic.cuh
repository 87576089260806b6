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
    void *Ps = nullptr;  // kK1Prep only: P also in the BF16 split operand layout
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

// The multi-band analytic signal (k_bands.cu), one instantiation per
// (Tin, operand precision); T = 2^log2T with kMinLog2Bands <= log2T <= 13.
template <typename Tin, int PREC>
cudaError_t launch_bands(const Handle *h, cudaStream_t st, const Tin *x, int64_t ldx, int N,
                         int64_t rows, int log2T, const float *masks, int nbands, void *P,
                         int64_t band_bytes);
#define PLV_BANDS_EXTERN(TIN, KIND)                                                           \
    extern template cudaError_t launch_bands<TIN, KIND>(const Handle *, cudaStream_t,        \
                                                        const TIN *, int64_t, int, int64_t,  \
                                                        int, const float *, int, void *,     \
                                                        int64_t);
PLV_BANDS_EXTERN(float, kK1Fp32)
PLV_BANDS_EXTERN(double, kK1Fp32)
PLV_BANDS_EXTERN(float, kK1Bf16)
PLV_BANDS_EXTERN(double, kK1Bf16)
PLV_BANDS_EXTERN(float, kK1Fp16)
PLV_BANDS_EXTERN(double, kK1Fp16)
#undef PLV_BANDS_EXTERN

// The multi-band analytic signal for any other T up to kMaxConvM / 2
// (k_bands.cu): one row per transform of length M, the forward spectrum kept
// in `scratch` (per CTA, M complex values), per band a multiply by K_b
// ([nbands][M]) and an inverse transform.  scratch must hold
// bands_conv_scratch(h, M) complex values.
template <typename Tin, int PREC>
cudaError_t launch_bands_conv(const Handle *h, cudaStream_t st, const Tin *x, int64_t ldx,
                              int N, int64_t rows, int T, const ConvPlan &plan, const float2 *K,
                              int nbands, void *P, int64_t band_bytes, float2 *scratch);
#define PLV_BANDS_CONV_EXTERN(TIN, KIND)                                                      \
    extern template cudaError_t launch_bands_conv<TIN, KIND>(                                 \
        const Handle *, cudaStream_t, const TIN *, int64_t, int, int64_t, int,                \
        const ConvPlan &, const float2 *, int, void *, int64_t, float2 *);
PLV_BANDS_CONV_EXTERN(float, kK1Fp32)
PLV_BANDS_CONV_EXTERN(double, kK1Fp32)
PLV_BANDS_CONV_EXTERN(float, kK1Bf16)
PLV_BANDS_CONV_EXTERN(double, kK1Bf16)
PLV_BANDS_CONV_EXTERN(float, kK1Fp16)
PLV_BANDS_CONV_EXTERN(double, kK1Fp16)
#undef PLV_BANDS_CONV_EXTERN

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
    if (!PLV_IN_BOUNDS(m >= 0 && m < ld)) return;
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

// Eight consecutive samples m0 .. m0+7 (m0 a multiple of 8) of a row of x.
template <typename Tin>
__device__ __forceinline__ void load_x8(const Tin *p, float (&v)[8]) {
    if constexpr (sizeof(Tin) == 4) {
        if (((uintptr_t)p & 15) == 0) {
            const float4 a = __ldg((const float4 *)p), b = __ldg((const float4 *)p + 1);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
            return;
        }
    } else {
        if (((uintptr_t)p & 15) == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double2 a = __ldg((const double2 *)p + k);
                v[2 * k] = (float)a.x;
                v[2 * k + 1] = (float)a.y;
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = ldx_f(p + k);
}

// Two 16-bit values (a at the lower address) as one 32-bit word, with the
// rounding of the per-sample store: hi = RN(p), lo = RN(p - hi).
template <int PREC>
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    if constexpr (PREC == PLV_PREC_FP16X3) {
        const __half2 h = __floats2half2_rn(a, b);
        const __half2 l = __floats2half2_rn(a - __low2float(h), b - __high2float(h));
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const __nv_bfloat162 l =
            __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}

// Store eight consecutive phasors m0 .. m0+7 of a row (m0 a multiple of 8):
// FP32, two 16-byte stores per plane; split layout, one 16-byte chunk (the
// eight samples of one swizzled chunk of the row) per plane.  Same values
// as eight store_phasor calls.
template <int PREC>
__device__ __forceinline__ void store_phasor8(void *P, const RowAddr<PREC> &ra, int64_t ld,
                                              int m0, const float2 (&p)[8]) {
    if (!PLV_IN_BOUNDS(m0 >= 0 && (m0 & 7) == 0 && m0 + 8 <= ld)) return;
    if constexpr (PREC == PLV_PREC_FP32) {
        float4 *o = (float4 *)((float *)P + ra.base + m0);
        o[0] = make_float4(p[0].x, p[1].x, p[2].x, p[3].x);
        o[1] = make_float4(p[4].x, p[5].x, p[6].x, p[7].x);
        float4 *q = (float4 *)((float *)P + ra.base + ld + m0);
        q[0] = make_float4(p[0].y, p[1].y, p[2].y, p[3].y);
        q[1] = make_float4(p[4].y, p[5].y, p[6].y, p[7].y);
    } else {
        const int64_t off = ra.base + (int64_t)(m0 >> 5) * kBlockElems +
                            ((((m0 & 31) >> 3) ^ ra.sw) << 3);
        constexpr int64_t ps = kTileRows * kTileK;  // plane stride in a block
        uint4 rh, rl, ih, il;
        split2<PREC>(p[0].x, p[1].x, rh.x, rl.x);
        split2<PREC>(p[2].x, p[3].x, rh.y, rl.y);
        split2<PREC>(p[4].x, p[5].x, rh.z, rl.z);
        split2<PREC>(p[6].x, p[7].x, rh.w, rl.w);
        split2<PREC>(p[0].y, p[1].y, ih.x, il.x);
        split2<PREC>(p[2].y, p[3].y, ih.y, il.y);
        split2<PREC>(p[4].y, p[5].y, ih.z, il.z);
        split2<PREC>(p[6].y, p[7].y, ih.w, il.w);
        uint16_t *o = (uint16_t *)P + off;
        *(uint4 *)o = rh;
        *(uint4 *)(o + ps) = rl;
        *(uint4 *)(o + 2 * ps) = ih;
        *(uint4 *)(o + 3 * ps) = il;
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
    // L2 prefetch of rows r0, r1 (the power-of-two engine issues it one
    // pair's work ahead)
    static constexpr bool kPrefetch = true;
    __device__ void prefetch(int64_t r0, bool v0, int64_t r1, bool v1) const {
        const uint32_t bytes = (uint32_t)(ld * sizeof(Tin)) <= (uint32_t)(ldx * sizeof(Tin))
                                   ? (uint32_t)(ld * sizeof(Tin)) : (uint32_t)(ldx * sizeof(Tin));
        if (v0) prefetch_l2(x + r0 * ldx, bytes);
        if (v1) prefetch_l2(x + r1 * ldx, bytes);
    }
    // one Newton step on 1/|z| except for the BF16 split
    static constexpr bool kNewton = PREC != PLV_PREC_BF16X3;
    __device__ void finish(const Rows &rs, int m, float h0, float h1, float floor2) const {
        if (rs.x0)
            store_phasor<PREC>(P, rs.a0, ld, m, unit_phasor<kNewton>(ldx_f(rs.x0 + m), h0, floor2));
        if (rs.x1)
            store_phasor<PREC>(P, rs.a1, ld, m, unit_phasor<kNewton>(ldx_f(rs.x1 + m), h1, floor2));
    }
    // finish() for eight consecutive samples m0 .. m0+7 < ld (m0 % 8 == 0)
    static constexpr bool kFinish8 = true;
    __device__ void row8(const Tin *xr, const RowAddr<PREC> &ra, int m0, const float (&h)[8],
                         float floor2) const {
        float xv[8];
        load_x8(xr + m0, xv);
        float2 p[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) p[k] = unit_phasor<kNewton>(xv[k], h[k], floor2);
        store_phasor8<PREC>(P, ra, ld, m0, p);
    }
    __device__ void finish8(const Rows &rs, int m0, const float (&h0)[8], const float (&h1)[8],
                            float floor2) const {
        if (rs.x0) row8(rs.x0, rs.a0, m0, h0, floor2);
        if (rs.x1) row8(rs.x1, rs.a1, m0, h1, floor2);
    }
    // padding samples T <= m < ld are zero
    __device__ void pad(const Rows &rs, int m) const {
        if (rs.x0) store_phasor<PREC>(P, rs.a0, ld, m, make_float2(0.f, 0.f));
        if (rs.x1) store_phasor<PREC>(P, rs.a1, ld, m, make_float2(0.f, 0.f));
    }
};

// Backward preparation: the same analytic signal, stored as FP32 phasors
// P[row][2][ld] and the reciprocal amplitude rinv[row][ld] = 1/|z| (0 where
// |z| counts as 0), which the gradient of Eq. 4 needs; with SPLIT also as
// BF16 hi + lo splits in the tiled operand layout at Ps (rows of N per
// epoch), the B operand of the tensor-core contraction.
template <typename Tin, bool SPLIT = false>
struct PrepTask {
    const Tin *x;
    int64_t ldx;
    float *P;
    float *rinv;
    int64_t ld;
    void *Ps;
    int N;
    struct Rows {
        const Tin *x0, *x1;
        float *p0, *p1, *q0, *q1;  // phasor rows, reciprocal-amplitude rows
        RowAddr<PLV_PREC_BF16X3> s0, s1;  // SPLIT: rows of the split layout
    };
    __device__ Rows rows(int64_t r0, bool v0, int64_t r1, bool v1) const {
        Rows rs;
        rs.x0 = v0 ? x + r0 * ldx : nullptr;
        rs.x1 = v1 ? x + r1 * ldx : nullptr;
        rs.p0 = P + (v0 ? r0 : 0) * 2 * ld;
        rs.p1 = P + (v1 ? r1 : 0) * 2 * ld;
        rs.q0 = rinv + (v0 ? r0 : 0) * ld;
        rs.q1 = rinv + (v1 ? r1 : 0) * ld;
        if constexpr (SPLIT) {
            rs.s0 = row_addr<PLV_PREC_BF16X3>(v0 ? r0 : 0, N, ld);
            rs.s1 = row_addr<PLV_PREC_BF16X3>(v1 ? r1 : 0, N, ld);
        }
        return rs;
    }
    __device__ void one(const Tin *xr, float *pr, float *qr, const RowAddr<PLV_PREC_BF16X3> &sa,
                        int m, float h, float floor2) const {
        float ri;
        const float2 p = unit_phasor_inv(ldx_f(xr + m), h, floor2, ri);
        pr[m] = p.x;
        pr[ld + m] = p.y;
        qr[m] = ri;
        if constexpr (SPLIT) store_phasor<PLV_PREC_BF16X3>(Ps, sa, ld, m, p);
    }
    __device__ float2 load(const Rows &rs, int m) const {
        return make_float2(rs.x0 ? ldx_f(rs.x0 + m) : 0.f, rs.x1 ? ldx_f(rs.x1 + m) : 0.f);
    }
    __device__ void finish(const Rows &rs, int m, float h0, float h1, float floor2) const {
        if (rs.x0) one(rs.x0, rs.p0, rs.q0, rs.s0, m, h0, floor2);
        if (rs.x1) one(rs.x1, rs.p1, rs.q1, rs.s1, m, h1, floor2);
    }
    // eight consecutive samples m0 .. m0+7 (m0 % 8 == 0, m0 + 8 <= ld):
    // vector loads of x and 16-byte stores of both planes and of 1/|z|
    static constexpr bool kFinish8 = true;
    __device__ void row8(const Tin *xr, float *pr, float *qr, const RowAddr<PLV_PREC_BF16X3> &sa,
                         int m0, const float (&h)[8], float floor2) const {
        if (!PLV_IN_BOUNDS(m0 >= 0 && (m0 & 7) == 0 && m0 + 8 <= ld)) return;
        float xv[8];
        load_x8(xr + m0, xv);
        float2 p[8];
        float ri[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) p[k] = unit_phasor_inv(xv[k], h[k], floor2, ri[k]);
        float4 *o = (float4 *)(pr + m0), *oi = (float4 *)(pr + ld + m0), *oq = (float4 *)(qr + m0);
        o[0] = make_float4(p[0].x, p[1].x, p[2].x, p[3].x);
        o[1] = make_float4(p[4].x, p[5].x, p[6].x, p[7].x);
        oi[0] = make_float4(p[0].y, p[1].y, p[2].y, p[3].y);
        oi[1] = make_float4(p[4].y, p[5].y, p[6].y, p[7].y);
        oq[0] = make_float4(ri[0], ri[1], ri[2], ri[3]);
        oq[1] = make_float4(ri[4], ri[5], ri[6], ri[7]);
        if constexpr (SPLIT) store_phasor8<PLV_PREC_BF16X3>(Ps, sa, ld, m0, p);
    }
    __device__ void finish8(const Rows &rs, int m0, const float (&h0)[8], const float (&h1)[8],
                            float floor2) const {
        if (rs.x0) row8(rs.x0, rs.p0, rs.q0, rs.s0, m0, h0, floor2);
        if (rs.x1) row8(rs.x1, rs.p1, rs.q1, rs.s1, m0, h1, floor2);
    }
    static constexpr bool kPrefetch = true;
    __device__ void prefetch(int64_t r0, bool v0, int64_t r1, bool v1) const {
        const uint32_t bytes = (uint32_t)(ld * sizeof(Tin)) <= (uint32_t)(ldx * sizeof(Tin))
                                   ? (uint32_t)(ld * sizeof(Tin)) : (uint32_t)(ldx * sizeof(Tin));
        if (v0) prefetch_l2(x + r0 * ldx, bytes);
        if (v1) prefetch_l2(x + r1 * ldx, bytes);
    }
    __device__ void pad(const Rows &rs, int m) const {
        if (rs.x0) { rs.p0[m] = 0.f; rs.p0[ld + m] = 0.f; rs.q0[m] = 0.f; }
        if (rs.x1) { rs.p1[m] = 0.f; rs.p1[ld + m] = 0.f; rs.q1[m] = 0.f; }
        if constexpr (SPLIT) {
            if (rs.x0) store_phasor<PLV_PREC_BF16X3>(Ps, rs.s0, ld, m, make_float2(0.f, 0.f));
            if (rs.x1) store_phasor<PLV_PREC_BF16X3>(Ps, rs.s1, ld, m, make_float2(0.f, 0.f));
        }
    }
};

}  // namespace
}  // namespace plv
