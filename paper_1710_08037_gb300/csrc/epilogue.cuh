// epilogue.cuh -- the Gram epilogue shared by the SIMT and the tensor-core
// kernels: read-outs of one Gram entry written to (i, j) and mirrored to
// (j, i), plus the FP64 unit-modulus check of the diagonal.
#pragma once

#include "common.cuh"
#include "readout.cuh"

namespace plv {

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
    // for non-negative doubles the IEEE bit pattern orders like an integer
    atomicMax((unsigned long long *)addr,
              (unsigned long long)__double_as_longlong(v));
}

// Write the read-outs of C_ij (already scaled by 1/T) to (i, j) and their
// mirror to (j, i): PLV and iPLV symmetric, ciPLV negated, C conjugated.
// On the diagonal Im C_ii = sum_t |P_i|^2 / T is real: it is stored as 0 and
// iPLV = ciPLV = 0 there.
__device__ __forceinline__ void emit(const GramOut &o, int64_t eNN, int N,
                                     int i, int j, float re, float im) {
    if (!PLV_IN_BOUNDS(i >= 0 && j >= 0 && i < N && j < N)) return;
    const int64_t ij = eNN + (int64_t)i * N + j;
    const int64_t ji = eNN + (int64_t)j * N + i;
    float p, ip, cp;
    if (i == j) {
        im = 0.f;
        p = plv_of(re, im);
        ip = 0.f;
        cp = 0.f;
    } else {
        readout(re, im, p, ip, cp);
    }
    if (o.plv) { o.plv[ij] = p; if (i != j) o.plv[ji] = p; }
    if (o.iplv) { o.iplv[ij] = ip; if (i != j) o.iplv[ji] = ip; }
    if (o.ciplv) { o.ciplv[ij] = cp; if (i != j) o.ciplv[ji] = -cp; }
    if (o.C) {
        o.C[ij] = make_float2(re, im);
        if (i != j) o.C[ji] = make_float2(re, -im);
    }
}

// max_i |C_ii - 1| with the 1/T applied in FP64 (the unit-modulus check of
// Eq. 4: |P| = 1 makes C_ii = 1 exactly in exact arithmetic).
__device__ __forceinline__ void diag_check(double *diag, float acc_re,
                                           float acc_im, double invT_d) {
    const double dr = (double)acc_re * invT_d - 1.0;
    const double di = (double)acc_im * invT_d;
    atomic_max_nonneg(diag, sqrt(dr * dr + di * di));
}

// One thread's W consecutive Gram sums of row i, columns j0 .. j0+W-1, of an
// upper-triangle tile (unscaled accumulators): scale by 1/T, read-outs,
// direct store along the row (16-byte vector stores where the row segment is
// complete and aligned) and mirrored store to (j, i).  Within a warp the
// lanes hold consecutive rows i, so every mirrored store is one coalesced
// segment.  On a diagonal tile only i <= j is stored (its mirror covers the
// rest).
template <int W>
__device__ __forceinline__ void store_tile_row(const GramOut &o, int64_t eNN, int N,
                                               int i, int j0, bool diag_tile,
                                               const float (&sre)[W],
                                               const float (&sim)[W], float invT,
                                               double invT_d, double *diag) {
    const bool row_ok = i < N;
    const bool vec = o.vec_ok && row_ok && !diag_tile && (j0 + W <= N);
    const int64_t rowbase = eNN + (int64_t)i * N;
#pragma unroll
    for (int g = 0; g < W / 4; ++g) {
        float p[4], ip[4], cp[4], rr[4], mm[4];
        bool valid[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int jj = 4 * g + u;
            const int j = j0 + jj;
            valid[u] = row_ok && j < N && (!diag_tile || i <= j);
            float re = sre[jj] * invT, im = sim[jj] * invT;
            if (i == j) {
                if (valid[u] && diag) diag_check(diag, sre[jj], sim[jj], invT_d);
                im = 0.f;
                p[u] = plv_of(re, im);
                ip[u] = 0.f;
                cp[u] = 0.f;
            } else {
                readout(re, im, p[u], ip[u], cp[u]);
            }
            rr[u] = re;
            mm[u] = im;
        }
        const int64_t d0 = rowbase + j0 + 4 * g;
        if (vec) {
            if (o.plv) *(float4 *)(o.plv + d0) = make_float4(p[0], p[1], p[2], p[3]);
            if (o.iplv) *(float4 *)(o.iplv + d0) = make_float4(ip[0], ip[1], ip[2], ip[3]);
            if (o.ciplv) *(float4 *)(o.ciplv + d0) = make_float4(cp[0], cp[1], cp[2], cp[3]);
            if (o.C) {
                float4 *c4 = (float4 *)(o.C + d0);
                c4[0] = make_float4(rr[0], mm[0], rr[1], mm[1]);
                c4[1] = make_float4(rr[2], mm[2], rr[3], mm[3]);
            }
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!valid[u]) continue;
                if (o.plv) o.plv[d0 + u] = p[u];
                if (o.iplv) o.iplv[d0 + u] = ip[u];
                if (o.ciplv) o.ciplv[d0 + u] = cp[u];
                if (o.C) o.C[d0 + u] = make_float2(rr[u], mm[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + 4 * g + u;
            if (!valid[u] || i == j) continue;
            const int64_t m = eNN + (int64_t)j * N + i;
            if (o.plv) o.plv[m] = p[u];
            if (o.iplv) o.iplv[m] = ip[u];
            if (o.ciplv) o.ciplv[m] = -cp[u];
            if (o.C) o.C[m] = make_float2(rr[u], -mm[u]);
        }
    }
}

// One metric of an off-diagonal Gram entry (re, im already scaled): the same
// arithmetic as readout(), so both store paths give identical bits.
__device__ __forceinline__ float metric_of(int m, float re, float im) {
    if (m == 0) return plv_of(re, im);
    if (m == 1) return fabsf(im);
    return ciplv_of(re, im);
}

// One metric m of one 8-column quarter (columns j0 .. j0+7, values re[c],
// im[c] unscaled) of a warp's 32 x 32 block: the mirrored and the staged
// row-wise stores described below.
__device__ __forceinline__ void store_block8(const GramOut &o, int m, int64_t eNN, int N,
                                             int i0, int j0, int lane, const float *re,
                                             const float *im, float invT, float *S, bool vec) {
    float *out = m == 0 ? o.plv : (m == 1 ? o.iplv : o.ciplv);
    if (!out) return;
    // checked builds: the whole 32 x 8 block lies inside the N x N matrix
    if (!PLV_IN_BOUNDS(i0 >= 0 && j0 >= 0 && i0 + 32 <= N && j0 + 8 <= N)) return;
    const float sgn = m == 2 ? -1.0f : 1.0f;  // ciPLV is antisymmetric
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = metric_of(m, re[c] * invT, im[c] * invT);
#pragma unroll
    for (int c = 0; c < 8; ++c) out[eNN + (int64_t)(j0 + c) * N + i0 + lane] = sgn * v[c];
    __syncwarp();  // the previous round's reads of S are done
    const int sw = (lane >> 2) & 1;
    *(float4 *)(S + lane * 8 + 4 * sw) = make_float4(v[0], v[1], v[2], v[3]);
    *(float4 *)(S + lane * 8 + 4 * (1 ^ sw)) = make_float4(v[4], v[5], v[6], v[7]);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int r = 16 * k + (lane >> 1), qq = lane & 1;
        const float4 w = *(const float4 *)(S + r * 8 + 4 * (qq ^ ((r >> 2) & 1)));
        float *d = out + eNN + (int64_t)(i0 + r) * N + j0 + 4 * qq;
        if (vec) {
            *(float4 *)d = w;
        } else {
            d[0] = w.x;
            d[1] = w.y;
            d[2] = w.z;
            d[3] = w.w;
        }
    }
}

// The store of one warp's 32 x 32 block of an interior off-diagonal tile:
// lane l holds row i0 + l, columns j0 .. j0+31 (unscaled sums).  Every row
// and column of the block is in range (the caller checks; the condition is
// warp-uniform).  With vec (N % 4 == 0, outputs 16-byte aligned) the
// row-wise segments are written as 16-byte vectors, else as four floats.
// Per metric and per 8-column quarter:
//   - mirrored store (j, i) straight from registers: for each column the
//     warp writes 32 consecutive floats (one 128-byte line);
//   - row-wise store through the warp's 32 x 8 staging tile S (1 KB; the
//     16-byte chunk q of row r sits at chunk q ^ ((r >> 2) & 1), so writes
//     and reads are free of bank conflicts): each instruction writes 16 rows
//     x 32 contiguous bytes (whole sectors) instead of 32 rows x 16 bytes.
__device__ __forceinline__ void store_tile_staged(const GramOut &o, int64_t eNN, int N, int i0,
                                                  int j0, int lane, const float (&sre)[32],
                                                  const float (&sim)[32], float invT,
                                                  float *S, bool vec) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
#pragma unroll
        for (int h = 0; h < 4; ++h)
            store_block8(o, m, eNN, N, i0, j0 + 8 * h, lane, sre + 8 * h, sim + 8 * h, invT, S,
                         vec);
    }
}

}  // namespace plv
