// k_dft.cu -- the DFT of real rows at F selected bins (the Fourier
// coefficients X(f) of Eq. 10-12 that coherency across trials is built
// from): X[r][f] = sum_t x[r][t] exp(-2 pi i (f0 + f) t / T).
//
// For a handful of bins this is a thin real GEMM (rows x T) . (T x 2F), so
// it runs on the CUDA cores: a CTA takes 128 rows and up to 32 bins, and
// walks t in tiles of 32.  Per tile the x block (128 x 32) and the tile's
// twiddles (32 x F, sincospif of the exact phase index ((f0 + f) t) mod T,
// which fits 32 bits for T <= 32768) are staged in shared memory; every
// thread accumulates a 4-row x 4-bin complex block.  Two-level summation: each tile's 32 terms are summed into
// a fresh register and then added to the running sum, so the rounding grows
// with 32 + T/32 terms rather than T.
#include "common.cuh"

namespace plv {
namespace {

constexpr int DR = 128;   // rows per CTA
constexpr int DK = 32;    // samples per tile
constexpr int DFMAX = 32; // bins per launch: 8 warps x 4 bins (the host splits larger F)

template <typename Tin>
__global__ void __launch_bounds__(256)
k_dft_bins(const Tin *__restrict__ x, int64_t rows, int T, int64_t ldx, int f0, int F,
           float *__restrict__ X, int64_t ldX) {
    __shared__ float xs[DK][DR + 4];            // [t][row]
    __shared__ float2 ws[DK][DFMAX];            // [t][bin] = (cos, -sin)
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * DR;
    // thread block: rows rb*4 .. +3 (rb = tid & 31), bins fb*4 .. +3 (fb = tid >> 5)
    const int rb = tid & 31, fb = tid >> 5;
    float ar[4][4], ai[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) { ar[a][c] = 0.f; ai[a][c] = 0.f; }
    const bool active = fb * 4 < F;
    for (int t0 = 0; t0 < T; t0 += DK) {
        __syncthreads();  // the previous tile has been consumed
        // x tile: 128 rows x 32 samples, lanes along t
        for (int q = tid; q < DR * DK; q += 256) {
            const int rr = q >> 5, tt = q & 31;
            const int64_t r = r0 + rr;
            const int t = t0 + tt;
            xs[tt][rr] = (r < rows && t < T) ? (float)__ldg(&x[r * ldx + t]) : 0.f;
        }
        // twiddles of the tile; the phase index is reduced exactly in integers
        for (int q = tid; q < DK * F; q += 256) {
            const int tt = q / F, f = q - tt * F;
            const int t = t0 + tt;
            const unsigned m = ((unsigned)(f0 + f) * (unsigned)t) % (unsigned)T;
            float s, c;
            sincospif((float)(2 * m) / (float)T, &s, &c);
            ws[tt][f] = make_float2(c, -s);
        }
        __syncthreads();
        if (active) {
            float pr[4][4], pi[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) { pr[a][c] = 0.f; pi[a][c] = 0.f; }
#pragma unroll 4
            for (int tt = 0; tt < DK; ++tt) {
                const float4 xv = *(const float4 *)&xs[tt][rb * 4];
                const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
                float2 w[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int f = fb * 4 + c;
                    w[c] = f < F ? ws[tt][f] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        pr[a][c] = fmaf(xa[a], w[c].x, pr[a][c]);
                        pi[a][c] = fmaf(xa[a], w[c].y, pi[a][c]);
                    }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    ar[a][c] += pr[a][c];
                    ai[a][c] += pi[a][c];
                }
        }
    }
    if (!active) return;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t r = r0 + rb * 4 + a;
        if (r >= rows) continue;
        float *o = X + r * 2 * ldX;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int f = fb * 4 + c;
            if (f >= F) continue;
            o[f] = ar[a][c];
            o[ldX + f] = ai[a][c];
        }
    }
}

}  // namespace

cudaError_t launch_dft_bins(cudaStream_t s, const void *x, plv_dtype dt, int64_t rows, int T,
                            int64_t ldx, int f0, int F, float *X, int64_t ldX) {
    for (int fs = 0; fs < F; fs += DFMAX) {
        const int Fc = F - fs < DFMAX ? F - fs : DFMAX;
        const int64_t blocks = (rows + DR - 1) / DR;
        if (blocks == 0) return cudaSuccess;
        if (dt == PLV_F32)
            k_dft_bins<float><<<(unsigned)blocks, 256, 0, s>>>((const float *)x, rows, T, ldx,
                                                               f0 + fs, Fc, X + fs, ldX);
        else
            k_dft_bins<double><<<(unsigned)blocks, 256, 0, s>>>((const double *)x, rows, T, ldx,
                                                                f0 + fs, Fc, X + fs, ldX);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace plv
