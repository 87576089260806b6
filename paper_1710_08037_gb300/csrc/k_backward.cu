// k_backward.cu -- K5: gradient of L = sum_ij (g_plv PLV + g_iplv iPLV +
// g_ciplv ciPLV)_ij with respect to the real input signals x, through the
// read-outs (Eq. 7, 13, 14), the Gram (Eq. 7), the normalisation (Eq. 4) and
// the analytic signal (Eq. 3).
//
// With R = Re C, I = Im C and d = (1 - R)(1 + R):
//   G_ij = dL/dR_ij + i dL/dI_ij,
//     dL/dR = g_plv R/|C| + g_ciplv I R / d^(3/2),
//     dL/dI = g_plv I/|C| + g_iplv sign(I) + g_ciplv / d^(1/2)
//   (each term only where the forward read-out is differentiable and
//   nonzero: |C| > 0, d > 0; the diagonal, whose forward values do not
//   depend on x, contributes nothing).
//   dL = Re sum conj(Gamma_P) dP with Gamma_P = (G + G^H) P / T = S P / T.
//   P = z/|z|:  Gamma_z = i P Im(conj(P) Gamma_P) / |z|.
//   z = A x with A = IFFT diag(h) FFT Hermitian (real part identity, imaginary
//   part the Hilbert transform H, H^T = -H):
//     dL/dx = Re Gamma_z - H{Im Gamma_z}.
//
// Stages:
//   1. recompute P and 1/|z| from x (the forward FFT task, fft.cuh), FP32,
//      and for split-precision handles P's BF16 splits in the operand layout;
//   2. S = G + G^H from C and the upstream gradients, 32x32 tiles staged
//      through shared memory for the transposed reads;
//   3. Gamma = S P / T, the one dense contraction of the pass:
//      - FP32 handles: k_bwd_gemm on the CUDA cores.  S is Hermitian, so
//        Gamma[i][t] = sum_k conj(S[k][i]) P[k][t] / T and both operands are
//        read as rows (no transposes): 128x128 tiles, 8x8 complex register
//        blocks, double-buffered shared memory;
//      - split-precision handles: the tensor-core kernel of the Gram in its
//        GEMM mode (BF16 hi + lo splits, three products per term).  Stage 2
//        then writes S as split rows (k_bwd_s_split, K-major A operand) and
//        the MMA reads stage 1's split P rows (row k, t contiguous) as an
//        MN-major B operand, so P is never transposed;
//   4. BwdTask on the FFT engine: u = -Im(P) s, v = Re(P) s with
//      s = Im(conj(P) Gamma) / |z|, then grad = u - H{v}.
#include "fft.cuh"
#include "readout.cuh"

namespace plv {
namespace {

using namespace fft;

__device__ __forceinline__ float2 gfun(float2 c, float g1, float g2, float g3) {
    const float R = c.x, I = c.y;
    float a = 0.f, b = 0.f;
    if (g1 != 0.f) {
        const float mag = sqrtf(fmaf(R, R, I * I));
        if (mag > 0.f) {
            a = fmaf(g1, R / mag, a);
            b = fmaf(g1, I / mag, b);
        }
    }
    if (g2 != 0.f) b += I > 0.f ? g2 : (I < 0.f ? -g2 : 0.f);
    if (g3 != 0.f) {
        const float d = ciplv_den(R);
        if (d > 0.f) {
            const float sd = sqrtf(d);
            b += g3 / sd;
            a += g3 * I * R / (d * sd);
        }
    }
    return make_float2(a, b);
}

// S = G + G^H for one epoch tile pair; S planar [B][2][N][N].
__global__ void __launch_bounds__(256)
k_bwd_s(const float2 *__restrict__ C, const float *__restrict__ g1,
        const float *__restrict__ g2, const float *__restrict__ g3, int N,
        float *__restrict__ S) {
    __shared__ float2 Gt[32][33];
    const int b = blockIdx.z;
    const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t NN = (int64_t)N * N;
    const int64_t eb = (int64_t)b * NN;
    auto G = [&](int r, int c) -> float2 {
        if (r >= N || c >= N || r == c) return make_float2(0.f, 0.f);
        const int64_t q = eb + (int64_t)r * N + c;
        return gfun(C[q], g1 ? g1[q] : 0.f, g2 ? g2[q] : 0.f, g3 ? g3[q] : 0.f);
    };
    // G of the transposed tile: Gt[yy][tx] = G(bj + yy, bi + tx)
    for (int yy = ty; yy < 32; yy += 8) Gt[yy][tx] = G(bj + yy, bi + tx);
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const int i = bi + yy, j = bj + tx;
        if (i >= N || j >= N) continue;
        const float2 gij = G(i, j);
        const float2 gji = Gt[tx][yy];  // G(j, i)
        const int64_t q = (int64_t)b * 2 * NN + (int64_t)i * N + j;
        S[q] = gij.x + gji.x;       // Re(G_ij + conj(G_ji))
        S[q + NN] = gij.y - gji.y;  // Im
    }
}

// One complex value as BF16 hi + lo splits at plane-0 element `off` of the
// tiled split layout (planes Re_hi, Re_lo, Im_hi, Im_lo, kTileRows x kTileK
// elements apart).
__device__ __forceinline__ void store_split_bf16(__nv_bfloat16 *base, int64_t off, float2 v) {
    constexpr int64_t ps = kTileRows * kTileK;
    const __nv_bfloat16 rh = __float2bfloat16_rn(v.x);
    const __nv_bfloat16 ih = __float2bfloat16_rn(v.y);
    base[off] = rh;
    base[off + ps] = __float2bfloat16_rn(v.x - __bfloat162float(rh));
    base[off + 2 * ps] = ih;
    base[off + 3 * ps] = __float2bfloat16_rn(v.y - __bfloat162float(ih));
}

// S = G + G^H as the A operand of the tensor-core contraction: row i, K = k,
// tiled split layout with NRB row blocks and NKB blocks of 32 along k.  S is
// Hermitian, so one block takes the pair of 32 x 32 tiles (p, q) and (q, p),
// p <= q: it forms G once on both, S(p, q) = G(p, q) + G(q, p)^H, and writes
// S(p, q) and its conjugate transpose S(q, p).  Rows and columns from N up
// to the 32-tile edge are zeros (G is 0 there), so the zero columns k >= N
// meet the B operand's zero rows.  The 128-row padding past the last 32-row
// tile is not written: it only feeds output rows i >= N, which are never
// stored.
__global__ void __launch_bounds__(256)
k_bwd_s_split(const float2 *__restrict__ C, const float *__restrict__ g1,
              const float *__restrict__ g2, const float *__restrict__ g3, int N, int64_t NRB,
              int64_t NKB, __nv_bfloat16 *__restrict__ A) {
    __shared__ float2 Gt[32][33];  // G(q-tile rows, p-tile columns), transposed on read
    __shared__ float2 Sm[32][33];  // S(p, q)
    const int b = blockIdx.y;
    // pair index -> (p, q), p <= q, column-major over the upper triangle
    const int t = blockIdx.x;
    int q = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((q + 1) * (q + 2) / 2 <= t) ++q;
    while (q * (q + 1) / 2 > t) --q;
    const int p = t - q * (q + 1) / 2;
    const int bi = p * 32, bk = q * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t eb = (int64_t)b * N * N;
    // the inputs of both tiles are loaded before any G is formed, so that
    // each thread has its 8 loads of C (and of the gradients) in flight at once
    float2 cv[8];
    float a1[8], a2[8], a3[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        // u < 4: (k, i) of the transposed tile; u >= 4: (i, k)
        const int yy = ty + 8 * (u & 3);
        const int r = u < 4 ? bk + yy : bi + yy, c = u < 4 ? bi + tx : bk + tx;
        const bool ok = r < N && c < N && r != c;
        const int64_t qq = eb + (int64_t)(ok ? r : 0) * N + (ok ? c : 0);
        cv[u] = ok ? __ldg(C + qq) : make_float2(0.f, 0.f);
        a1[u] = ok && g1 ? __ldg(g1 + qq) : 0.f;
        a2[u] = ok && g2 ? __ldg(g2 + qq) : 0.f;
        a3[u] = ok && g3 ? __ldg(g3 + qq) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) Gt[ty + 8 * u][tx] = gfun(cv[u], a1[u], a2[u], a3[u]);  // G(k, i)
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int yy = ty + 8 * u;
        const float2 gik = gfun(cv[4 + u], a1[4 + u], a2[4 + u], a3[4 + u]);
        const float2 gki = Gt[tx][yy];
        const float2 v = make_float2(gik.x + gki.x, gik.y - gki.y);  // G_ik + conj(G_ki)
        Sm[yy][tx] = v;
        store_split_bf16(A, split_offset(b, bi + yy, bk + tx, NRB, NKB), v);
    }
    if (p == q) return;  // the diagonal pair is its own mirror
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const float2 v = Sm[tx][yy];  // S(bi + tx, bk + yy)
        store_split_bf16(A, split_offset(b, bk + yy, bi + tx, NRB, NKB), make_float2(v.x, -v.y));
    }
}

constexpr int BM = 128, BK = 8;

// Gamma[b][i][plane][t] = (1/T) sum_k conj(S[b][k][i]) P[b][k][plane][t].
__global__ void __launch_bounds__(256, 1)
k_bwd_gemm(const float *__restrict__ S, const float *__restrict__ P, int N, int64_t ld,
           float invT, float *__restrict__ Gm) {
    __shared__ __align__(16) float As[2][2][BK][BM];
    __shared__ __align__(16) float Bs[2][2][BK][BM];
    const int b = blockIdx.z;
    const int i0 = blockIdx.y * BM;
    const int64_t t0 = (int64_t)blockIdx.x * BM;
    const int64_t NN = (int64_t)N * N;
    const float *Sr = S + (int64_t)b * 2 * NN;
    const float *Si = Sr + NN;
    const float *Pb = P + (int64_t)b * N * 2 * ld;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int lk = tid >> 5, lc = (tid & 31) * 4;  // loader: row k, 4 columns
    const bool vi = i0 + lc < N;                   // N % 4 may be nonzero: per element
    const bool vt = t0 + lc < ld;

    float cre[8][8], cim[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) { cre[a][c] = 0.f; cim[a][c] = 0.f; }

    auto ld_s = [&](const float *base, int k) -> float4 {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < N && vi) {
            const float *p = base + (int64_t)k * N + i0 + lc;
            v.x = p[0];
            if (i0 + lc + 1 < N) v.y = p[1];
            if (i0 + lc + 2 < N) v.z = p[2];
            if (i0 + lc + 3 < N) v.w = p[3];
        }
        return v;
    };
    auto ld_p = [&](int k, int plane) -> float4 {
        if (k < N && vt)
            return __ldg((const float4 *)(Pb + ((int64_t)k * 2 + plane) * ld + t0 + lc));
        return make_float4(0.f, 0.f, 0.f, 0.f);
    };
    float4 sr = ld_s(Sr, lk), si = ld_s(Si, lk), pr = ld_p(lk, 0), pi = ld_p(lk, 1);
    auto stash = [&](int st) {
        *(float4 *)&As[st][0][lk][lc] = sr;
        *(float4 *)&As[st][1][lk][lc] = si;
        *(float4 *)&Bs[st][0][lk][lc] = pr;
        *(float4 *)&Bs[st][1][lk][lc] = pi;
    };
    stash(0);
    __syncthreads();
    const int nk = (N + BK - 1) / BK;
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt + 1 < nk) {
            const int k = (kt + 1) * BK + lk;
            sr = ld_s(Sr, k);
            si = ld_s(Si, k);
            pr = ld_p(k, 0);
            pi = ld_p(k, 1);
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
                for (int c = 0; c < 8; ++c) {
                    // conj(s) p = (sr pr + si pi) + i (sr pi - si pr)
                    cre[a][c] = fmaf(a_r[a], b_r[c], cre[a][c]);
                    cre[a][c] = fmaf(a_i[a], b_i[c], cre[a][c]);
                    cim[a][c] = fmaf(a_r[a], b_i[c], cim[a][c]);
                    cim[a][c] = fmaf(-a_i[a], b_r[c], cim[a][c]);
                }
        }
        if (kt + 1 < nk) stash(st ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int i = i0 + (a < 4 ? ty * 4 + a : 64 + ty * 4 + a - 4);
        if (i >= N) continue;
        float *gr = Gm + ((int64_t)b * N + i) * 2 * ld;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t t = t0 + (h == 0 ? tx * 4 : 64 + tx * 4);
            if (t >= ld) continue;
            *(float4 *)(gr + t) = make_float4(cre[a][4 * h] * invT, cre[a][4 * h + 1] * invT,
                                              cre[a][4 * h + 2] * invT, cre[a][4 * h + 3] * invT);
            *(float4 *)(gr + ld + t) =
                make_float4(cim[a][4 * h] * invT, cim[a][4 * h + 1] * invT,
                            cim[a][4 * h + 2] * invT, cim[a][4 * h + 3] * invT);
        }
    }
}

// Stage 4 on the FFT engine: rows of v = Re(P) s in, grad = -Im(P) s - H{v}
// out, s = Im(conj(P) Gamma) / |z|.
struct BwdTask {
    // load() forms u, v from P, Gamma and 1/|z| (see below)
    static constexpr bool kLoadComputes = true;
    const float *P;     // [rows][2][ld]
    const float *Gm;    // [rows][2][ld]
    const float *rinv;  // [rows][ld]
    float *grad;        // [rows][T]
    int64_t ld;
    int T;
    struct Row {
        const float *p, *g, *q;
        float *o;
    };
    struct Rows {
        Row a, b;
        bool v0, v1;
    };
    __device__ Row row(int64_t r) const {
        return Row{P + r * 2 * ld, Gm + r * 2 * ld, rinv + r * ld, grad + r * T};
    }
    __device__ Rows rows(int64_t r0, bool v0, int64_t r1, bool v1) const {
        return Rows{row(v0 ? r0 : 0), row(v1 ? r1 : 0), v0, v1};
    }
    __device__ float s_of(const Row &w, int m, float &pr, float &pi) const {
        pr = w.p[m];
        pi = w.p[ld + m];
        return fmaf(pr, w.g[ld + m], -pi * w.g[m]) * w.q[m];
    }
    __device__ float2 load(const Rows &rs, int m) const {
        float pr, pi, a = 0.f, b = 0.f;
        if (rs.v0) a = s_of(rs.a, m, pr, pi) * pr;
        if (rs.v1) b = s_of(rs.b, m, pr, pi) * pr;
        return make_float2(a, b);
    }
    __device__ void pad(const Rows &, int) const {}  // grad has no padding
    // eight consecutive samples m0 .. m0+7 (m0 % 8 == 0): 16-byte loads of P,
    // Gamma and 1/|z| and 16-byte stores of grad (rows are 32-float aligned)
    static constexpr bool kFinish8 = true;
    __device__ void row8(const Row &w, int m0, const float (&h)[8]) const {
        if (!PLV_IN_BOUNDS(m0 >= 0 && (m0 & 7) == 0 && m0 + 8 <= T)) return;
        float pr[8], pi[8], gr[8], gi[8], q[8];
        auto ld8 = [](const float *p, float (&v)[8]) {
            const float4 a = __ldg((const float4 *)p), b = __ldg((const float4 *)p + 1);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        };
        ld8(w.p + m0, pr);
        ld8(w.p + ld + m0, pi);
        ld8(w.g + m0, gr);
        ld8(w.g + ld + m0, gi);
        ld8(w.q + m0, q);
        float o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float sk = fmaf(pr[k], gi[k], -pi[k] * gr[k]) * q[k];
            o[k] = -pi[k] * sk - h[k];
        }
        float4 *d = (float4 *)(w.o + m0);
        d[0] = make_float4(o[0], o[1], o[2], o[3]);
        d[1] = make_float4(o[4], o[5], o[6], o[7]);
    }
    __device__ void finish8(const Rows &rs, int m0, const float (&h0)[8], const float (&h1)[8],
                            float) const {
        if (rs.v0) row8(rs.a, m0, h0);
        if (rs.v1) row8(rs.b, m0, h1);
    }
    __device__ void finish(const Rows &rs, int m, float h0, float h1, float) const {
        float pr, pi;
        if (rs.v0) {
            const float s = s_of(rs.a, m, pr, pi);
            rs.a.o[m] = -pi * s - h0;
        }
        if (rs.v1) {
            const float s = s_of(rs.b, m, pr, pi);
            rs.b.o[m] = -pi * s - h1;
        }
    }
};

}  // namespace

size_t backward_tc_bytes(int batch, int N, int T, size_t *a_bytes) {
    const int64_t NKB = ((int64_t)N + kTileK - 1) / kTileK;
    const size_t a = (size_t)batch * row_blocks(N) * NKB * kBlockElems * 2;
    const size_t b = (size_t)batch * row_blocks(N) * (padded_len(T) / kTileK) * kBlockElems * 2;
    if (a_bytes) *a_bytes = a;
    return a + b;
}

cudaError_t launch_backward(const Handle *h, cudaStream_t st, int batch, int N, int T,
                            int log2T, const float2 *C, const float *g1, const float *g2,
                            const float *g3, const float *P, const float *rinv, float *S,
                            float *Gm, float *grad, const ConvPlan *plan, void *tc_a,
                            const void *tc_b) {
    const int64_t ld = padded_len(T);
    cudaError_t e;
    if (tc_a) {
        // S as split rows, then the contraction on the tensor cores
        if (!tc_b) return cudaErrorInvalidValue;
        __nv_bfloat16 *A = (__nv_bfloat16 *)tc_a;
        const uint8_t *B = (const uint8_t *)tc_b;  // stage 1 wrote it
        const int64_t NRB = row_blocks(N), NKB = ((int64_t)N + kTileK - 1) / kTileK;
        const int64_t NRBT = (ld + 127) / 128;  // output tiles along t
        const unsigned nt = (unsigned)NKB;  // 32-tiles along i and along k
        dim3 sg(nt * (nt + 1) / 2, batch);
        k_bwd_s_split<<<sg, 256, 0, st>>>(C, g1, g2, g3, N, NRB, NKB, A);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        TcGemm g;
        g.A = (const uint8_t *)A;
        g.B = B;
        g.nrb_a = (int)NRB;
        g.nrb_b = (int)NRBT;
        g.nkb = (int)NKB;
        g.nkb_t = (int)(ld / kTileK);
        g.tpe = (int)(NRB * NRBT);
        g.N = N;
        g.ld = ld;
        g.invT = 1.0f / (float)T;
        g.G = Gm;
        e = launch_gemm_tc(h, st, g, batch);
        if (e != cudaSuccess) return e;
    } else {
        dim3 sg((N + 31) / 32, (N + 31) / 32, batch);
        k_bwd_s<<<sg, 256, 0, st>>>(C, g1, g2, g3, N, S);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dim3 gg((unsigned)((ld + BM - 1) / BM), (N + BM - 1) / BM, batch);
        k_bwd_gemm<<<gg, 256, 0, st>>>(S, P, N, ld, 1.0f / (float)T, Gm);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    BwdTask task{P, Gm, rinv, grad, ld, T};
    if (plan) return launch_hilbert_conv(h->num_sms, st, task, *plan, T, ld, (int64_t)batch * N);
    return launch_hilbert_pow2(h->num_sms, st, log2T, task, twiddle_table(h, log2T),
                               (int64_t)batch * N);
}

}  // namespace plv
