// k_analytic.cu -- K1: the analytic signal (Eq. 3) by a shared-memory FFT,
// fused with the unit-phasor normalisation (Eq. 4) and the store in the
// Gram's operand layout.
//
// The Hilbert transform is a real-linear operator, so one complex FFT serves
// two real rows: with c = x1 + i x2,
//     w = IFFT(-i sgn(k) FFT(c)) = H{x1} + i H{x2},
// and the analytic signals are z1 = x1 + i Re w, z2 = x2 + i Im w (the real
// part of the discrete analytic signal equals the input exactly, because the
// analytic mask satisfies h[k] + h[-k] = 2).  The inverse transform is done
// with the forward one: IFFT(W) = conj(FFT(conj(W))) / T, and conj(W) is
// folded into the last forward pass.
//
// FFT: Stockham auto-sort (Govindaraju et al., SC'08) in shared memory,
// radix-16 passes plus one smaller radix for the remaining factor.  Every
// thread holds 16 elements; a sequence of T samples is served by T/16
// threads.  The first pass reads straight from global memory and the last
// inverse pass leaves each thread with the samples t = lt + u T/16 (u < 16),
// which makes both the input loads and the phasor stores coalesced.
// Shared-memory indices are padded by one element per 32 to spread banks.
#include "common.cuh"

namespace plv {
namespace {

__device__ __forceinline__ int padi(int i) { return i + (i >> 5); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    return make_float2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    return make_float2(a.x - b.x, a.y - b.y);
}
// a * w with w = (c, s) meaning c + i s
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}

// a * exp(-i pi m / 8), m in 0..7 (folds to a constant path after unrolling)
__device__ __forceinline__ float2 rot16(float2 a, int m) {
    const float c1 = 0.92387953251128675613f;  // cos(pi/8)
    const float s1 = 0.38268343236508977173f;  // sin(pi/8)
    const float h = 0.70710678118654752440f;   // cos(pi/4)
    switch (m) {
        case 0: return a;
        case 1: return make_float2(fmaf(a.x, c1, a.y * s1), fmaf(a.y, c1, -a.x * s1));
        case 2: return make_float2((a.x + a.y) * h, (a.y - a.x) * h);
        case 3: return make_float2(fmaf(a.x, s1, a.y * c1), fmaf(a.y, s1, -a.x * c1));
        case 4: return make_float2(a.y, -a.x);
        case 5: return make_float2(fmaf(-a.x, s1, a.y * c1), fmaf(-a.y, s1, -a.x * c1));
        case 6: return make_float2((a.y - a.x) * h, -(a.x + a.y) * h);
        default: return make_float2(fmaf(-a.x, c1, a.y * s1), fmaf(-a.y, c1, -a.x * s1));
    }
}

// In-register forward DFT of length R (R = 2, 4, 8, 16), natural order in
// and out: radix-2 decimation in time, recursively.
template <int R>
struct Dft {
    __device__ __forceinline__ static void run(float2 (&a)[R]) {
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            e[k] = a[2 * k];
            o[k] = a[2 * k + 1];
        }
        Dft<R / 2>::run(e);
        Dft<R / 2>::run(o);
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            const float2 t = rot16(o[k], (16 / R) * k);
            a[k] = cadd(e[k], t);
            a[k + R / 2] = csub(e[k], t);
        }
    }
};
template <>
struct Dft<1> {
    __device__ __forceinline__ static void run(float2 (&)[1]) {}
};

// Pass schedule for T = 2^L: 16 first, then the remainder radix 2^(L mod 4)
// if any, then radix-16 passes.  For L < 8 the schedule is [16, 2^(L-4)].
__host__ __device__ constexpr int npasses(int L) {
    return L / 4 + (L % 4 != 0 ? 1 : 0);
}
__host__ __device__ constexpr int radix_of(int L, int p) {
    return (p == 0) ? 16 : ((p == 1 && (L % 4) != 0) ? (1 << (L % 4)) : 16);
}
__host__ __device__ constexpr int ns_of(int L, int p) {
    return p == 0 ? 1 : ns_of(L, p - 1) * radix_of(L, p - 1);
}

enum PassMode { kSmem = 0, kFromX = 1, kToHilbert = 2, kToRegs = 3 };

template <typename Tin>
__device__ __forceinline__ float ldx_f(const Tin *p) {
    return (float)__ldg(p);
}

// One Stockham pass of radix R over the sequence in `s`.  NS is the length
// of the sub-transforms already formed.  MODE selects where the inputs come
// from and where the outputs go (see PassMode).  In kToRegs mode the output
// for sample lt + u*T/16 ends in out[u].
template <int T, int R, int NS, int MODE, typename Tin>
__device__ __forceinline__ void stockham(float2 *s, const float2 *__restrict__ tw,
                                         int lt, const Tin *x0, const Tin *x1,
                                         float2 (&out)[16], float *power = nullptr) {
    constexpr int B = 16 / R;  // butterflies per thread
    constexpr int Q = T / 16;  // threads per sequence
    float2 v[16];
    float pw = 0.f;
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int j = lt + q * Q;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = j + r * (T / R);
            if constexpr (MODE == kFromX) {
                const float2 c = make_float2(x0 ? ldx_f(x0 + m) : 0.f,
                                             x1 ? ldx_f(x1 + m) : 0.f);
                v[q * R + r] = c;
                pw = fmaf(c.x, c.x, fmaf(c.y, c.y, pw));
            } else {
                v[q * R + r] = s[padi(m)];
            }
        }
    }
    if constexpr (MODE != kFromX) __syncthreads();
    if constexpr (MODE == kFromX) *power = pw;
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int j = lt + q * Q;
        const int k = j & (NS - 1);
        float2 a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = v[q * R + r];
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r)
                a[r] = cmul(a[r], __ldg(&tw[r * k * (T / (NS * R))]));
        }
        Dft<R>::run(a);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = base + r * NS;
            if constexpr (MODE == kToRegs) {
                out[q + B * r] = a[r];
            } else if constexpr (MODE == kToHilbert) {
                // conj(-i sgn(m) C[m]) = sgn(m) (Im C, Re C)
                const float sg = (m == 0 || m == T / 2) ? 0.f
                                 : (m < T / 2 ? 1.f : -1.f);
                s[padi(m)] = make_float2(sg * a[r].y, sg * a[r].x);
            } else {
                s[padi(m)] = a[r];
            }
        }
    }
    if constexpr (MODE != kToRegs) __syncthreads();
}

// Middle passes p in [P, PEND) (shared memory to shared memory).
template <int L, int P, int PEND, typename Tin>
__device__ __forceinline__ void middle_passes(float2 *s, const float2 *tw,
                                              int lt, float2 (&dummy)[16]) {
    if constexpr (P < PEND) {
        stockham<(1 << L), radix_of(L, P), ns_of(L, P), kSmem, Tin>(
            s, tw, lt, (const Tin *)nullptr, (const Tin *)nullptr, dummy);
        middle_passes<L, P + 1, PEND, Tin>(s, tw, lt, dummy);
    }
}

// Unit phasor of z = a + i b (Eq. 4); |z|^2 <= floor2 (|z| = 0 by default)
// gives 0.  Very small or very large magnitudes are rescaled by a power of
// two first so the squared norm neither underflows nor overflows.
__device__ __forceinline__ float2 unit_phasor(float a, float b, float floor2 = 0.0f) {
    float r2 = fmaf(a, a, b * b);
    if (!(r2 > floor2)) return make_float2(0.f, 0.f);
    if (r2 < 1e-30f || r2 > 1e30f) {
        const float sc = r2 < 1e-30f ? 0x1p+60f : 0x1p-60f;
        a *= sc;
        b *= sc;
        r2 = fmaf(a, a, b * b);
    }
    const float inv = 1.0f / sqrtf(r2);
    return make_float2(a * inv, b * inv);
}

// Store one unit phasor of row r at sample m in the operand layout.
template <int PREC>
__device__ __forceinline__ void store_phasor(void *P, int64_t r, int N,
                                             int64_t ld, int m, float2 p) {
    if constexpr (PREC == PLV_PREC_FP32) {
        float *o = (float *)P + r * 2 * ld + m;
        o[0] = p.x;
        o[ld] = p.y;
    } else if constexpr (PREC == PLV_PREC_FP16X3) {
        const int64_t e = r / N, n = r - e * N;
        __half *o = (__half *)P + ((e * 4) * N + n) * ld + m;
        const int64_t ps = (int64_t)N * ld;  // plane stride
        const __half rh = __float2half_rn(p.x);
        const __half ih = __float2half_rn(p.y);
        o[0] = rh;
        o[ps] = __float2half_rn(p.x - __half2float(rh));
        o[2 * ps] = ih;
        o[3 * ps] = __float2half_rn(p.y - __half2float(ih));
    } else {
        const int64_t e = r / N, n = r - e * N;
        __nv_bfloat16 *o = (__nv_bfloat16 *)P + ((e * 4) * N + n) * ld + m;
        const int64_t ps = (int64_t)N * ld;  // plane stride
        const __nv_bfloat16 rh = __float2bfloat16_rn(p.x);
        const __nv_bfloat16 ih = __float2bfloat16_rn(p.y);
        o[0] = rh;
        o[ps] = __float2bfloat16_rn(p.x - __bfloat162float(rh));
        o[2 * ps] = ih;
        o[3 * ps] = __float2bfloat16_rn(p.y - __bfloat162float(ih));
    }
}

template <int L>
struct K1Cfg {
    static constexpr int T = 1 << L;
    static constexpr int Q = T / 16;                  // threads / sequence
    static constexpr int SEQ = Q >= 256 ? 1 : 256 / Q;  // sequences / CTA
    static constexpr int THREADS = Q * SEQ;
    static constexpr int SMEM_SEQ = T + T / 32;         // padded elements
    static constexpr size_t SMEM =
        (size_t)SEQ * SMEM_SEQ * sizeof(float2) + (size_t)SEQ * sizeof(float);
    // resident CTAs per SM the register budget is sized for
    static constexpr int MIN_BLOCKS = THREADS <= 256 ? 2 : 1;
};

template <int L, typename Tin, int PREC>
__global__ void __launch_bounds__(K1Cfg<L>::THREADS, K1Cfg<L>::MIN_BLOCKS)
k_analytic_pow2(const Tin *__restrict__ x, int64_t rows, int N, int64_t ldx,
                void *__restrict__ P, const float2 *__restrict__ tw) {
    using C = K1Cfg<L>;
    constexpr int T = C::T;
    constexpr int NP = npasses(L);
    extern __shared__ float2 smem[];
    const int lt = threadIdx.x % C::Q;
    const int sq = threadIdx.x / C::Q;
    float2 *s = smem + sq * C::SMEM_SEQ;
    const int64_t pair = (int64_t)blockIdx.x * C::SEQ + sq;
    const int64_t r0 = 2 * pair, r1 = 2 * pair + 1;
    const Tin *x0 = r0 < rows ? x + r0 * ldx : nullptr;
    const Tin *x1 = r1 < rows ? x + r1 * ldx : nullptr;
    float2 out[16];
    float *s_pow = (float *)(smem + C::SEQ * C::SMEM_SEQ);  // per-sequence power
    if (lt == 0) s_pow[sq] = 0.f;
    __syncthreads();

    // forward FFT of c = x0 + i x1
    float pw;
    stockham<T, radix_of(L, 0), 1, kFromX, Tin>(s, tw, lt, x0, x1, out, &pw);
    // sum of x0^2 + x1^2 over the sequence (its lanes are an aligned group of
    // Q threads, or whole warps when Q >= 32)
#pragma unroll
    for (int off = 1; off < (C::Q < 32 ? C::Q : 32); off <<= 1)
        pw += __shfl_xor_sync(0xffffffffu, pw, off);
    if ((lt & 31) == 0) atomicAdd(&s_pow[sq], pw);
    middle_passes<L, 1, NP - 1, Tin>(s, tw, lt, out);
    stockham<T, radix_of(L, NP - 1), ns_of(L, NP - 1), kToHilbert, Tin>(
        s, tw, lt, x0, x1, out);
    // inverse FFT (as a forward FFT of the conjugate) of -i sgn(k) C[k]
    stockham<T, radix_of(L, 0), 1, kSmem, Tin>(s, tw, lt, x0, x1, out);
    middle_passes<L, 1, NP - 1, Tin>(s, tw, lt, out);
    stockham<T, radix_of(L, NP - 1), ns_of(L, NP - 1), kToRegs, Tin>(
        s, tw, lt, x0, x1, out);

    constexpr float invT = 1.0f / (float)T;
    const int64_t ld = T;  // power-of-two T >= 32 needs no padding
    // |z|^2 below 2^-40 of the pair's mean power is under the FFT's rounding
    // (the two rows of a sequence leak into each other at that level): such
    // a sample carries no phase and is treated as |z| = 0.
    const float floor2 = 0x1p-40f * (s_pow[sq] * invT);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int m = lt + u * C::Q;
        const float h0 = out[u].x * invT;   // H{x0}[m]
        const float h1 = -out[u].y * invT;  // H{x1}[m]
        if (x0) store_phasor<PREC>(P, r0, N, ld, m, unit_phasor(ldx_f(x0 + m), h0, floor2));
        if (x1) store_phasor<PREC>(P, r1, N, ld, m, unit_phasor(ldx_f(x1 + m), h1, floor2));
    }
}

template <int L, typename Tin, int PREC>
cudaError_t launch_l(cudaStream_t st, const Tin *x, int64_t rows, int N,
                     int64_t ldx, void *P, const float2 *tw) {
    using C = K1Cfg<L>;
    auto kern = k_analytic_pow2<L, Tin, PREC>;
    if (C::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(
            kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t pairs = (rows + 1) / 2;
    const int64_t grid = (pairs + C::SEQ - 1) / C::SEQ;
    kern<<<(unsigned)grid, C::THREADS, C::SMEM, st>>>(x, rows, N, ldx, P, tw);
    return cudaGetLastError();
}

template <typename Tin, int PREC>
cudaError_t launch_t(cudaStream_t st, const Tin *x, int64_t rows, int N,
                     int log2T, int64_t ldx, void *P, const float2 *tw) {
    switch (log2T) {
        case 5: return launch_l<5, Tin, PREC>(st, x, rows, N, ldx, P, tw);
        case 6: return launch_l<6, Tin, PREC>(st, x, rows, N, ldx, P, tw);
        case 7: return launch_l<7, Tin, PREC>(st, x, rows, N, ldx, P, tw);
        case 8: return launch_l<8, Tin, PREC>(st, x, rows, N, ldx, P, tw);
        case 9: return launch_l<9, Tin, PREC>(st, x, rows, N, ldx, P, tw);
        case 10: return launch_l<10, Tin, PREC>(st, x, rows, N, ldx, P, tw);
        case 11: return launch_l<11, Tin, PREC>(st, x, rows, N, ldx, P, tw);
        case 12: return launch_l<12, Tin, PREC>(st, x, rows, N, ldx, P, tw);
        case 13: return launch_l<13, Tin, PREC>(st, x, rows, N, ldx, P, tw);
        case 14: return launch_l<14, Tin, PREC>(st, x, rows, N, ldx, P, tw);
        default: return cudaErrorInvalidValue;
    }
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
    store_phasor<PREC>(P, r, N, ld, (int)m, p);
}

}  // namespace

cudaError_t launch_analytic_pow2(const Handle *h, cudaStream_t s,
                                 const void *x, plv_dtype dt, int64_t rows,
                                 int N, int log2T, int64_t ldx, void *P) {
    const float2 *tw = twiddle_table(h, log2T);
    if (h->prec == PLV_PREC_FP32) {
        if (dt == PLV_F32)
            return launch_t<float, PLV_PREC_FP32>(s, (const float *)x, rows, N, log2T, ldx, P, tw);
        return launch_t<double, PLV_PREC_FP32>(s, (const double *)x, rows, N, log2T, ldx, P, tw);
    }
    if (h->prec == PLV_PREC_FP16X3) {
        if (dt == PLV_F32)
            return launch_t<float, PLV_PREC_FP16X3>(s, (const float *)x, rows, N, log2T, ldx, P, tw);
        return launch_t<double, PLV_PREC_FP16X3>(s, (const double *)x, rows, N, log2T, ldx, P, tw);
    }
    if (dt == PLV_F32)
        return launch_t<float, PLV_PREC_BF16X3>(s, (const float *)x, rows, N, log2T, ldx, P, tw);
    return launch_t<double, PLV_PREC_BF16X3>(s, (const double *)x, rows, N, log2T, ldx, P, tw);
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
