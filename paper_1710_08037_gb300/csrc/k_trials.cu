// k_trials.cu -- operands of a Gram over trials: the time-resolved PLV of
// Lachaux et al. (Eq. 1; Eq. 8 is its matrix form) and coherency across
// trials (Eq. 12) are the Hermitian Gram of Eq. 7 with the trials as the
// summation index, one problem per time sample (or frequency bin).
//
// Input: per-trial complex values as FP32 planar rows V[E][N][2][ldv] (the
// layout an FP32 handle's analytic-signal call writes).  Output: for every
// column l, the N x E operand whose row i is (V[0][i][l], ..., V[E-1][i][l]),
// in the handle's operand layout, so that the ordinary Gram with batch = L
// and T = E computes (1/E) sum_n P_i(n) conj(P_j(n)).  Mode RMS divides row
// (l, i) by sqrt(mean_n |V[n][i][l]|^2) first (the normalisation of Eq. 12),
// which makes that Gram the coherency.
//
// One CTA per (row i, 32 columns): the 32 x 32 (trial, column) tiles pass
// through shared memory, read along columns (coalesced in V) and written
// along trials (coalesced in the operand layout).
#include "analytic.cuh"

namespace plv {
namespace {

template <int PREC>
__device__ __forceinline__ void store_trial(void *P, int64_t l, int i, int n, int N,
                                            int64_t NRB, int64_t NKB, int64_t ldE, float2 v) {
    if constexpr (PREC == PLV_PREC_FP32) {
        float *o = (float *)P + ((l * N + i) * 2) * ldE + n;
        o[0] = v.x;
        o[ldE] = v.y;
    } else {
        constexpr int64_t ps = kTileRows * kTileK;
        const int64_t off = split_offset(l, i, n, NRB, NKB);
        if constexpr (PREC == PLV_PREC_FP16X3) {
            __half *o = (__half *)P + off;
            const __half rh = __float2half_rn(v.x), ih = __float2half_rn(v.y);
            o[0] = rh;
            o[ps] = __float2half_rn(v.x - __half2float(rh));
            o[2 * ps] = ih;
            o[3 * ps] = __float2half_rn(v.y - __half2float(ih));
        } else {
            __nv_bfloat16 *o = (__nv_bfloat16 *)P + off;
            const __nv_bfloat16 rh = __float2bfloat16_rn(v.x), ih = __float2bfloat16_rn(v.y);
            o[0] = rh;
            o[ps] = __float2bfloat16_rn(v.x - __bfloat162float(rh));
            o[2 * ps] = ih;
            o[3 * ps] = __float2bfloat16_rn(v.y - __bfloat162float(ih));
        }
    }
}

// Grid: x = ceil(L / 32) column tiles, y = operand rows (N, or the split
// layout's ceil(N/128)*128, whose padding rows are written as zeros).
// kpad: trials written per row (ld(E) for FP32, NKB * 32 for the split
// layout); trials E .. kpad-1 are zeros.
template <int PREC>
__global__ void __launch_bounds__(256)
k_trial_operands(const float *__restrict__ V, int E, int N, int64_t ldv, int l0, int L,
                 int rms, int64_t NRB, int64_t NKB, int64_t ldE, int kpad, void *P) {
    __shared__ float2 tile[32][33];  // [trial][column]
    __shared__ float red[8][33];
    __shared__ float scale[32];
    const int i = blockIdx.y;
    const int lb = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const bool col_ok = lb + tx < L;
    const bool row_ok = i < N;
    auto vat = [&](int n) -> float2 {
        const float *r = V + ((int64_t)n * N + i) * 2 * ldv + l0 + lb + tx;
        return make_float2(__ldg(r), __ldg(r + ldv));
    };
    float acc = 0.f;
    if (rms && row_ok && col_ok)
        for (int n = ty; n < E; n += 8) {
            const float2 v = vat(n);
            acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
        }
    red[ty][tx] = acc;
    __syncthreads();
    if (ty == 0) {
        float s = 1.f;
        if (rms) {
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) t += red[k][tx];
            s = t > 0.f ? sqrtf((float)E / t) : 0.f;
        }
        scale[tx] = s;
    }
    for (int n0 = 0; n0 < kpad; n0 += 32) {
        __syncthreads();  // scale is set; the previous tile has been written
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int n = n0 + ty + 8 * q;
            tile[ty + 8 * q][tx] =
                (row_ok && col_ok && n < E) ? vat(n) : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ll = ty + 8 * q;
            if (lb + ll >= L) continue;
            const float2 v = tile[tx][ll];
            const float s = scale[ll];
            store_trial<PREC>(P, (int64_t)lb + ll, i, n0 + tx, N, NRB, NKB, ldE,
                              make_float2(v.x * s, v.y * s));
        }
    }
}

}  // namespace

cudaError_t launch_trial_operands(const Handle *h, cudaStream_t s, const float *V, int E, int N,
                                  int64_t ldv, int l0, int L, int rms, void *P) {
    if (L == 0 || N == 0) return cudaSuccess;
    const int64_t ldE = padded_len(E);
    const int64_t NRB = row_blocks(N), NKB = ldE / kTileK;
    const bool split = h->prec != PLV_PREC_FP32;
    const int64_t rows = split ? NRB * kTileRows : N;
    dim3 grid((unsigned)((L + 31) / 32), (unsigned)rows);
    const int kpad = (int)ldE;
    if (h->prec == PLV_PREC_FP32)
        k_trial_operands<PLV_PREC_FP32><<<grid, 256, 0, s>>>(V, E, N, ldv, l0, L, rms, NRB, NKB,
                                                               ldE, kpad, P);
    else if (h->prec == PLV_PREC_FP16X3)
        k_trial_operands<PLV_PREC_FP16X3><<<grid, 256, 0, s>>>(V, E, N, ldv, l0, L, rms, NRB,
                                                                 NKB, ldE, kpad, P);
    else
        k_trial_operands<PLV_PREC_BF16X3><<<grid, 256, 0, s>>>(V, E, N, ldv, l0, L, rms, NRB,
                                                                 NKB, ldE, kpad, P);
    return cudaGetLastError();
}

}  // namespace plv
