// k_analytic.cu -- K1: the analytic signal (Eq. 3) by the shared-memory
// FFT engine (fft.cuh), fused with the unit-phasor normalisation (Eq. 4) and
// the store in the Gram's operand layout; and the recompute of P and 1/|z|
// that the backward pass starts from.
//
// The real part of the discrete analytic signal equals the input exactly
// (the analytic mask satisfies h[k] + h[-k] = 2), so z = x + i H{x} with H{x}
// from the engine and x re-read at the end (an L2 hit).
#include "fft.cuh"

namespace plv {
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

// Zero the rows N .. NRB*128-1 of every epoch's last row block, all planes
// and samples: one thread per 16-byte chunk.
__global__ void k_zero_pad_rows(uint4 *P, int batch, int N, int64_t NRB, int64_t NKB) {
    const int pad0 = N & 127;  // first padding row inside the last block
    const int npad = 128 - pad0;
    const int64_t chunks_per_row = kTileK * 2 / 16;  // 4 chunks of 16 bytes
    const int64_t per_block = 4 * (int64_t)npad * chunks_per_row;
    const int64_t total = (int64_t)batch * NKB * per_block;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = q % chunks_per_row;
        int64_t rest = q / chunks_per_row;
        const int64_t rr = rest % npad;
        rest /= npad;
        const int64_t plane = rest % 4;
        rest /= 4;
        const int64_t kb = rest % NKB;
        const int64_t e = rest / NKB;
        const int64_t blk = (e * NRB + (NRB - 1)) * NKB + kb;
        const int64_t el = blk * kBlockElems + plane * (kTileRows * kTileK) +
                           (pad0 + rr) * kTileK + c * 8;
        P[el / 8] = make_uint4(0u, 0u, 0u, 0u);
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

template <typename Tin, int PREC>
cudaError_t launch_fwd(const Handle *h, cudaStream_t st, const Tin *x, int64_t rows, int N,
                       int log2T, int64_t ldx, void *P, const float2 *tw) {
    FwdTask<Tin, PREC> task{x, ldx, P, N, (int64_t)1 << log2T};
    return launch_hilbert_pow2(h->num_sms, st, log2T, task, tw, rows);
}

// Eq. 4 on a caller-supplied analytic signal: one thread per padded sample.
template <typename Tc, int PREC>
__global__ void k_normalize(const Tc *__restrict__ z, int64_t rows, int N,
                            int T, int64_t ldz, int64_t ld, void *P) {
    const int64_t r = blockIdx.y + (int64_t)blockIdx.z * 65535;
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows || m >= ld) return;
    float2 p = make_float2(0.f, 0.f);
    if (m < T) {
        const Tc v = z[r * ldz + m];
        p = unit_phasor((float)v.x, (float)v.y);
    }
    store_phasor<PREC>(P, row_addr<PREC>(r, N, ld), ld, (int)m, p);
}

}  // namespace

cudaError_t launch_zero_pad_rows(cudaStream_t s, void *P, int batch, int N, int T) {
    if ((N & 127) == 0 || batch == 0) return cudaSuccess;
    const int64_t NKB = padded_len(T) / kTileK;
    const int64_t total = (int64_t)batch * NKB * 4 * (128 - (N & 127)) * 4;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_zero_pad_rows<<<(unsigned)blocks, 256, 0, s>>>((uint4 *)P, batch, N, row_blocks(N), NKB);
    return cudaGetLastError();
}

cudaError_t launch_analytic_conv(const Handle *h, cudaStream_t s, const void *x,
                                 plv_dtype dt, int64_t rows, int N, int T, int64_t ldx,
                                 void *P, const ConvPlan &plan) {
    const int64_t ld = padded_len(T);
    const int ns = h->num_sms;
    if (h->prec == PLV_PREC_FP32) {
        if (dt == PLV_F32)
            return launch_hilbert_conv(ns, s, FwdTask<float, PLV_PREC_FP32>{(const float *)x, ldx, P, N, ld}, plan, T, ld, rows);
        return launch_hilbert_conv(ns, s, FwdTask<double, PLV_PREC_FP32>{(const double *)x, ldx, P, N, ld}, plan, T, ld, rows);
    }
    if (h->prec == PLV_PREC_FP16X3) {
        if (dt == PLV_F32)
            return launch_hilbert_conv(ns, s, FwdTask<float, PLV_PREC_FP16X3>{(const float *)x, ldx, P, N, ld}, plan, T, ld, rows);
        return launch_hilbert_conv(ns, s, FwdTask<double, PLV_PREC_FP16X3>{(const double *)x, ldx, P, N, ld}, plan, T, ld, rows);
    }
    if (dt == PLV_F32)
        return launch_hilbert_conv(ns, s, FwdTask<float, PLV_PREC_BF16X3>{(const float *)x, ldx, P, N, ld}, plan, T, ld, rows);
    return launch_hilbert_conv(ns, s, FwdTask<double, PLV_PREC_BF16X3>{(const double *)x, ldx, P, N, ld}, plan, T, ld, rows);
}

cudaError_t launch_bwd_prep(const Handle *h, cudaStream_t s, const void *x, plv_dtype dt,
                            int64_t rows, int log2T, int64_t ldx, float *P, float *rinv,
                            int T, const ConvPlan *plan) {
    if (plan) {
        const int64_t ld = padded_len(T);
        if (dt == PLV_F32)
            return launch_hilbert_conv(h->num_sms, s, PrepTask<float>{(const float *)x, ldx, P, rinv, ld}, *plan, T, ld, rows);
        return launch_hilbert_conv(h->num_sms, s, PrepTask<double>{(const double *)x, ldx, P, rinv, ld}, *plan, T, ld, rows);
    }
    const float2 *tw = twiddle_table(h, log2T);
    const int64_t ld = (int64_t)1 << log2T;
    if (dt == PLV_F32) {
        PrepTask<float> task{(const float *)x, ldx, P, rinv, ld};
        return launch_hilbert_pow2(h->num_sms, s, log2T, task, tw, rows);
    }
    PrepTask<double> task{(const double *)x, ldx, P, rinv, ld};
    return launch_hilbert_pow2(h->num_sms, s, log2T, task, tw, rows);
}

cudaError_t launch_analytic_pow2(const Handle *h, cudaStream_t s,
                                 const void *x, plv_dtype dt, int64_t rows,
                                 int N, int log2T, int64_t ldx, void *P) {
    const float2 *tw = twiddle_table(h, log2T);
    if (h->prec == PLV_PREC_FP32) {
        if (dt == PLV_F32)
            return launch_fwd<float, PLV_PREC_FP32>(h, s, (const float *)x, rows, N, log2T, ldx, P, tw);
        return launch_fwd<double, PLV_PREC_FP32>(h, s, (const double *)x, rows, N, log2T, ldx, P, tw);
    }
    if (h->prec == PLV_PREC_FP16X3) {
        if (dt == PLV_F32)
            return launch_fwd<float, PLV_PREC_FP16X3>(h, s, (const float *)x, rows, N, log2T, ldx, P, tw);
        return launch_fwd<double, PLV_PREC_FP16X3>(h, s, (const double *)x, rows, N, log2T, ldx, P, tw);
    }
    if (dt == PLV_F32)
        return launch_fwd<float, PLV_PREC_BF16X3>(h, s, (const float *)x, rows, N, log2T, ldx, P, tw);
    return launch_fwd<double, PLV_PREC_BF16X3>(h, s, (const double *)x, rows, N, log2T, ldx, P, tw);
}

cudaError_t launch_normalize(const Handle *h, cudaStream_t s, const void *z,
                             plv_dtype dt, int64_t rows, int N, int T,
                             int64_t ldz, void *P) {
    const int64_t ld = padded_len(T);
    dim3 block(256);
    const int64_t gy = rows < 65535 ? rows : 65535;
    dim3 grid((unsigned)((ld + 255) / 256), (unsigned)gy,
              (unsigned)((rows + 65534) / 65535));
    if (h->prec == PLV_PREC_FP32) {
        if (dt == PLV_F32)
            k_normalize<float2, PLV_PREC_FP32><<<grid, block, 0, s>>>((const float2 *)z, rows, N, T, ldz, ld, P);
        else
            k_normalize<double2, PLV_PREC_FP32><<<grid, block, 0, s>>>((const double2 *)z, rows, N, T, ldz, ld, P);
    } else if (h->prec == PLV_PREC_FP16X3) {
        if (dt == PLV_F32)
            k_normalize<float2, PLV_PREC_FP16X3><<<grid, block, 0, s>>>((const float2 *)z, rows, N, T, ldz, ld, P);
        else
            k_normalize<double2, PLV_PREC_FP16X3><<<grid, block, 0, s>>>((const double2 *)z, rows, N, T, ldz, ld, P);
    } else {
        if (dt == PLV_F32)
            k_normalize<float2, PLV_PREC_BF16X3><<<grid, block, 0, s>>>((const float2 *)z, rows, N, T, ldz, ld, P);
        else
            k_normalize<double2, PLV_PREC_BF16X3><<<grid, block, 0, s>>>((const double2 *)z, rows, N, T, ldz, ld, P);
    }
    return cudaGetLastError();
}

}  // namespace plv
