// k_gram_simt.cu -- K2: the Hermitian Gram C = P P^H / T (Eq. 7) in plain
// FP32 on the CUDA cores, with the read-outs (Eq. 7, 13, 14) fused into the
// epilogue; and K6, the same read-outs from a stored C.
//
// One CTA computes one 128 x 128 tile (I, J), I <= J, of the upper triangle
// of one epoch; the tile is mirrored into the lower triangle by the same CTA,
// so PLV / iPLV come out exactly symmetric and ciPLV exactly antisymmetric.
// On a diagonal tile only the entries i <= j are computed into the output.
//
// Per sample t and pair (i, j), with P = a + i b:
//   Re C_ij += a_i a_j + b_i b_j,   Im C_ij += b_i a_j - a_i b_j.
// 256 threads, each owning an 8 x 8 block of complex accumulators; operands
// staged through double-buffered shared memory in [plane][k][row] order (the
// global layout is row-major in t, so the load transposes).
#include "epilogue.cuh"

namespace plv {
namespace {

constexpr int BM = 128;      // tile edge (rows of I and of J)
constexpr int BK = 8;        // samples per stage
constexpr int LDS = BM + 4;  // padded shared row (conflict-free transposed store)

// Output matrix e is window w = e % nw of epoch e / nw: samples t0 + w hop
// .. + kl (kl, t0, hop multiples of BK; one window of kl = ld for the whole
// epoch).
__global__ void __launch_bounds__(256, 1)
k_gram_fp32(const float *__restrict__ P, int N, int kl, int64_t ld,
            int tiles_per_epoch, GramOut out, float invT, double invT_d, int nw, int64_t t0,
            int64_t hop) {
    __shared__ __align__(16) float As[2][2][BK][LDS];
    __shared__ __align__(16) float Bs[2][2][BK][LDS];

    const int e = blockIdx.x / tiles_per_epoch;
    int I, J;
    upper_tile_of(blockIdx.x - e * tiles_per_epoch, I, J);
    const int eb = e / nw, w = e - eb * nw;
    const float *Pe = P + (int64_t)eb * N * 2 * ld + t0 + (int64_t)w * hop;

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    // loader: each thread moves 4 consecutive samples of one row, both planes
    const int lrow = tid >> 1, lk = (tid & 1) * 4;
    const int ga = I * BM + lrow, gb = J * BM + lrow;
    const float *pa = Pe + (int64_t)(ga < N ? ga : 0) * 2 * ld + lk;
    const float *pb = Pe + (int64_t)(gb < N ? gb : 0) * 2 * ld + lk;
    const bool va = ga < N, vb = gb < N;

    float cre[8][8], cim[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) { cre[a][b] = 0.f; cim[a][b] = 0.f; }

    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 ar = va ? __ldg((const float4 *)pa) : z4;
    float4 ai = va ? __ldg((const float4 *)(pa + ld)) : z4;
    float4 br = vb ? __ldg((const float4 *)pb) : z4;
    float4 bi = vb ? __ldg((const float4 *)(pb + ld)) : z4;

    auto stash = [&](int st) {
        As[st][0][lk + 0][lrow] = ar.x; As[st][0][lk + 1][lrow] = ar.y;
        As[st][0][lk + 2][lrow] = ar.z; As[st][0][lk + 3][lrow] = ar.w;
        As[st][1][lk + 0][lrow] = ai.x; As[st][1][lk + 1][lrow] = ai.y;
        As[st][1][lk + 2][lrow] = ai.z; As[st][1][lk + 3][lrow] = ai.w;
        Bs[st][0][lk + 0][lrow] = br.x; Bs[st][0][lk + 1][lrow] = br.y;
        Bs[st][0][lk + 2][lrow] = br.z; Bs[st][0][lk + 3][lrow] = br.w;
        Bs[st][1][lk + 0][lrow] = bi.x; Bs[st][1][lk + 1][lrow] = bi.y;
        Bs[st][1][lk + 2][lrow] = bi.z; Bs[st][1][lk + 3][lrow] = bi.w;
    };
    stash(0);
    __syncthreads();

    const int nk = kl / BK;
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt + 1 < nk) {
            const int64_t off = (int64_t)(kt + 1) * BK;
            ar = va ? __ldg((const float4 *)(pa + off)) : z4;
            ai = va ? __ldg((const float4 *)(pa + ld + off)) : z4;
            br = vb ? __ldg((const float4 *)(pb + off)) : z4;
            bi = vb ? __ldg((const float4 *)(pb + ld + off)) : z4;
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a_r[8], a_i[8], b_r[8], b_i[8];
            *(float4 *)&a_r[0] = *(const float4 *)&As[st][0][kk][ty * 4];
            *(float4 *)&a_r[4] = *(const float4 *)&As[st][0][kk][64 + ty * 4];
            *(float4 *)&a_i[0] = *(const float4 *)&As[st][1][kk][ty * 4];
            *(float4 *)&a_i[4] = *(const float4 *)&As[st][1][kk][64 + ty * 4];
            *(float4 *)&b_r[0] = *(const float4 *)&Bs[st][0][kk][tx * 4];
            *(float4 *)&b_r[4] = *(const float4 *)&Bs[st][0][kk][64 + tx * 4];
            *(float4 *)&b_i[0] = *(const float4 *)&Bs[st][1][kk][tx * 4];
            *(float4 *)&b_i[4] = *(const float4 *)&Bs[st][1][kk][64 + tx * 4];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    cre[a][b] = fmaf(a_r[a], b_r[b], cre[a][b]);
                    cre[a][b] = fmaf(a_i[a], b_i[b], cre[a][b]);
                    cim[a][b] = fmaf(a_i[a], b_r[b], cim[a][b]);
                    cim[a][b] = fmaf(-a_r[a], b_i[b], cim[a][b]);
                }
        }
        if (kt + 1 < nk) stash(st ^ 1);
        __syncthreads();
    }

    const int64_t eNN = (int64_t)e * N * N;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int i = I * BM + (a < 4 ? ty * 4 + a : 64 + ty * 4 + a - 4);
        if (i >= N) continue;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int j = J * BM + (b < 4 ? tx * 4 + b : 64 + tx * 4 + b - 4);
            if (j >= N || (I == J && i > j)) continue;
            emit(out, eNN, N, i, j, cre[a][b] * invT, cim[a][b] * invT);
            if (i == j && out.diag)
                diag_check(out.diag + e, cre[a][b], cim[a][b], invT_d);
        }
    }
}

__global__ void k_metrics(const float2 *__restrict__ C, int64_t total, int N,
                          float *plv, float *iplv, float *ciplv) {
    const int64_t NN = (int64_t)N * N;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const float2 c = C[q];
        const int64_t w = q % NN;
        const bool diag = (w / N) == (w % N);
        float p, ip, cp;
        if (diag) {
            p = plv_of(c.x, c.y);
            ip = 0.f;
            cp = 0.f;
        } else {
            readout(c.x, c.y, p, ip, cp);
        }
        if (plv) plv[q] = p;
        if (iplv) iplv[q] = ip;
        if (ciplv) ciplv[q] = cp;
    }
}

}  // namespace

cudaError_t launch_gram_fp32(const Handle *h, cudaStream_t s, const float *P,
                             int batch, int N, int T, GramOut out) {
    const int nt = (N + BM - 1) / BM;
    const int tiles = nt * (nt + 1) / 2;
    const int64_t grid = (int64_t)tiles * batch;
    if (grid > 0x7fffffff) return cudaErrorInvalidConfiguration;
    k_gram_fp32<<<(unsigned)grid, 256, 0, s>>>(P, N, (int)padded_len(T), padded_len(T), tiles,
                                               out, 1.0f / (float)T, 1.0 / (double)T, 1, 0, 0);
    return cudaGetLastError();
}

cudaError_t launch_gram_fp32_windows(const Handle *h, cudaStream_t s, const float *P, int batch,
                                     int N, int T, int t0, int W, int hop, int nw, GramOut out) {
    const int nt = (N + BM - 1) / BM;
    const int tiles = nt * (nt + 1) / 2;
    const int64_t grid = (int64_t)tiles * batch * nw;
    if (grid > 0x7fffffff) return cudaErrorInvalidConfiguration;
    if (grid == 0) return cudaSuccess;
    k_gram_fp32<<<(unsigned)grid, 256, 0, s>>>(P, N, W, padded_len(T), tiles, out,
                                               1.0f / (float)W, 1.0 / (double)W, nw, t0, hop);
    return cudaGetLastError();
}

cudaError_t launch_metrics(cudaStream_t s, const float2 *C, int batch, int N,
                           float *plv, float *iplv, float *ciplv) {
    const int64_t total = (int64_t)batch * N * N;
    if (total == 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_metrics<<<(unsigned)blocks, 256, 0, s>>>(C, total, N, plv, iplv, ciplv);
    return cudaGetLastError();
}

}  // namespace plv
