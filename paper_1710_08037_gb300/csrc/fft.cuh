// fft.cuh -- shared-memory FFT engine for the Hilbert transform of real rows
// (device code shared by the forward phasor kernel and the backward kernel).
//
// The Hilbert transform is a real-linear operator, so one complex FFT serves
// two real rows: with c = u0 + i u1,
//     w = IFFT(-i sgn(k) FFT(c)) = H{u0} + i H{u1}.
// The inverse transform is done with the forward one:
// IFFT(W) = conj(FFT(conj(W))) / T, and conj(W) is folded into the last
// forward pass.
//
// FFT: Stockham auto-sort (Govindaraju et al., SC'08) in shared memory,
// radix-16 passes plus one smaller radix for the remaining factor.  Every
// thread holds 16 elements; a sequence of T samples is served by T/16
// threads.  Shared-memory indices are padded by one element per 32 to spread
// banks.  Passes alternate between two shared buffers, so one barrier per
// pass separates a pass's reads from the next pass's writes.  The kernel is
// persistent over row pairs.
#pragma once

#include "common.cuh"

namespace plv {
namespace fft {

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

// Elements per thread of the power-of-two engine (its largest radix, R_E),
// and the registers per thread its launch bounds plan for.
constexpr int kPow2EPT = 16;
constexpr int kPow2LogEPT = kPow2EPT == 16 ? 4 : (kPow2EPT == 8 ? 3 : 2);
constexpr int kPow2Regs = 128;

// Pass schedule for T = 2^L: R_E first, then the remainder radix
// 2^(L mod log2 R_E) if any, then radix-R_E passes.
__host__ __device__ constexpr int npasses(int L) {
    return L / kPow2LogEPT + (L % kPow2LogEPT != 0 ? 1 : 0);
}
__host__ __device__ constexpr int radix_of(int L, int p) {
    return (p == 0) ? kPow2EPT
                    : ((p == 1 && (L % kPow2LogEPT) != 0) ? (1 << (L % kPow2LogEPT))
                                                          : kPow2EPT);
}
__host__ __device__ constexpr int ns_of(int L, int p) {
    return p == 0 ? 1 : ns_of(L, p - 1) * radix_of(L, p - 1);
}

enum PassMode { kSmem = 0, kFromX = 1, kToHilbert = 2 };

// Radix-16 passes of the power-of-two engine form their twiddles w^r from
// the table values w, w^2, w^4 and w^8 (4 loads instead of 15; the other
// powers are products of at most three, about one ulp each).  Measured 25 %
// faster at T = 4096.  (The any-length engine loads its few per-butterfly
// twiddles directly: there the same change measured no difference.)
constexpr bool kTwiddlePowers = true;

// One Stockham pass of radix R from shared buffer `src` to `dst` (distinct
// buffers, so no barrier is needed between this pass's reads and writes).
// NS is the length of the sub-transforms already formed.  MODE selects where
// the inputs come from (src, or load(m) for the first pass, which also sums
// |c|^2 into *power) and where the outputs go (dst, or dst with the analytic
// mask folded in).
template <int T, int R, int NS, int MODE, typename Load>
__device__ __forceinline__ void stockham(const float2 *src, float2 *dst,
                                         const float2 *__restrict__ tw, int lt,
                                         const Load &load, float *power = nullptr) {
    constexpr int B = kPow2EPT / R;  // butterflies per thread
    constexpr int Q = T / kPow2EPT;  // threads per sequence
    float pw = 0.f;
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int j = lt + q * Q;
        const int k = j & (NS - 1);
        float2 a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = j + r * (T / R);
            if constexpr (MODE == kFromX) {
                const float2 c = load(m);
                a[r] = c;
                pw = fmaf(c.x, c.x, fmaf(c.y, c.y, pw));
            } else {
                a[r] = src[padi(m)];
            }
        }
        if constexpr (NS > 1) {
            const int ts = k * (T / (NS * R));  // w = tw[ts]; a[r] *= w^r
            if constexpr (R == 16 && kTwiddlePowers) {
                // four loads (w, w^2, w^4, w^8); the other powers are products
                // of at most three of them, each product one more rounding
                float2 w[16];
                w[1] = __ldg(&tw[ts]);
                w[2] = __ldg(&tw[2 * ts]);
                w[4] = __ldg(&tw[4 * ts]);
                w[8] = __ldg(&tw[8 * ts]);
                w[3] = cmul(w[1], w[2]);
                w[5] = cmul(w[1], w[4]);
                w[6] = cmul(w[2], w[4]);
                w[7] = cmul(w[3], w[4]);
                w[9] = cmul(w[1], w[8]);
                w[10] = cmul(w[2], w[8]);
                w[11] = cmul(w[3], w[8]);
                w[12] = cmul(w[4], w[8]);
                w[13] = cmul(w[5], w[8]);
                w[14] = cmul(w[6], w[8]);
                w[15] = cmul(w[7], w[8]);
#pragma unroll
                for (int r = 1; r < R; ++r) a[r] = cmul(a[r], w[r]);
            } else {
#pragma unroll
                for (int r = 1; r < R; ++r) a[r] = cmul(a[r], __ldg(&tw[r * ts]));
            }
        }
        Dft<R>::run(a);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = base + r * NS;
            if constexpr (MODE == kToHilbert) {
                // conj(-i sgn(m) C[m]) = sgn(m) (Im C, Re C)
                const float sg = (m == 0 || m == T / 2) ? 0.f
                                 : (m < T / 2 ? 1.f : -1.f);
                dst[padi(m)] = make_float2(sg * a[r].y, sg * a[r].x);
            } else {
                dst[padi(m)] = a[r];
            }
        }
    }
    if constexpr (MODE == kFromX) *power = pw;
    __syncthreads();
}

// Passes p in [P, PEND), ping-ponging between the two buffers; pass p reads
// buffer (p & 1) and writes buffer (p & 1) ^ 1.
struct NoLoad {
    __device__ float2 operator()(int) const { return make_float2(0.f, 0.f); }
};

template <int L, int P, int PEND>
__device__ __forceinline__ void middle_passes(float2 *const (&buf)[2], const float2 *tw,
                                              int lt) {
    if constexpr (P < PEND) {
        stockham<(1 << L), radix_of(L, P), ns_of(L, P), kSmem>(
            buf[P & 1], buf[(P & 1) ^ 1], tw, lt, NoLoad{});
        middle_passes<L, P + 1, PEND>(buf, tw, lt);
    }
}

// Unit phasor of z = a + i b (Eq. 4); |z|^2 <= floor2 (|z| = 0 by default)
// gives 0.  Very small or very large magnitudes are rescaled by a power of
// two first so the squared norm neither underflows nor overflows.  1/|z| is
// the hardware reciprocal-square-root estimate (a few ulp), refined by one
// Newton step unless NEWTON is false: the BF16 hi + lo split keeps 2^-17 of
// a component, far coarser than the estimate's error.
template <bool NEWTON = true>
__device__ __forceinline__ float2 unit_phasor(float a, float b, float floor2 = 0.0f) {
    float r2 = fmaf(a, a, b * b);
    if (!(r2 > floor2)) return make_float2(0.f, 0.f);
    if (r2 < 1e-30f || r2 > 1e30f) {
        const float sc = r2 < 1e-30f ? 0x1p+60f : 0x1p-60f;
        a *= sc;
        b *= sc;
        r2 = fmaf(a, a, b * b);
    }
    float inv = rsqrtf(r2);
    if (NEWTON) inv = inv * fmaf(-0.5f * r2 * inv, inv, 1.5f);
    return make_float2(a * inv, b * inv);
}

// As unit_phasor, also returning rinv = 1/|z| (0 where the phasor is 0).
__device__ __forceinline__ float2 unit_phasor_inv(float a, float b, float floor2,
                                                  float &rinv) {
    float r2 = fmaf(a, a, b * b);
    rinv = 0.f;
    if (!(r2 > floor2)) return make_float2(0.f, 0.f);
    float sc = 1.0f;
    if (r2 < 1e-30f || r2 > 1e30f) {
        sc = r2 < 1e-30f ? 0x1p+60f : 0x1p-60f;
        a *= sc;
        b *= sc;
        r2 = fmaf(a, a, b * b);
    }
    float inv = rsqrtf(r2);
    inv = inv * fmaf(-0.5f * r2 * inv, inv, 1.5f);
    rinv = inv * sc;
    return make_float2(a * inv, b * inv);
}

// Tasks that also take eight consecutive samples at once (kFinish8).
template <class Task, class = void>
struct HasFinish8 {
    static constexpr bool value = false;
};
template <class Task>
struct HasFinish8<Task, decltype((void)Task::kFinish8)> {
    static constexpr bool value = Task::kFinish8;
};

// ---------------------------------------------------------------------------
// The power-of-two engine's kernel.
//
// Per row pair: forward passes 0 .. NP-1, then inverse passes 0 .. NP-1 (the
// inverse as a forward FFT of the conjugated, masked spectrum), then the
// task's finish.  The last forward pass (radix 16, NS = T/16, one butterfly
// per thread at j = lt) and the first inverse pass (radix 16, NS = 1, j = lt)
// touch the same 16 elements lt + r T/16 on the same thread, so for T >= 256
// they run fused in registers with the analytic mask between them: one
// shared-memory round trip and one barrier fewer per pair.  The mask
// conj(-i sgn(m) C[m]) / T = sgn(m) (Im C, Re C) / T also carries the 1/T of
// the inverse transform.
//
// The twiddles of every pass p >= 1 come from a table in shared memory,
// filled once per (persistent) CTA from the FP64-rounded global table:
// for each twiddle position k < NS and s < R/2 the pair
// (w^(2s ts), w^((2s+1) ts)), w = exp(-2 pi i / T), ts = k T / (NS R),
// as one float4 at tab_off(L, p) + s NS + k.  Consecutive k sit 16 bytes
// apart, so a warp's 16-byte reads are conflict-free.

__host__ __device__ constexpr int tab_len(int L, int p) {
    return (radix_of(L, p) / 2) * ns_of(L, p);
}
__host__ __device__ constexpr int tab_off(int L, int p) {
    return p <= 1 ? 0 : tab_off(L, p - 1) + tab_len(L, p - 1);
}

template <int L>
struct K1Cfg {
    static constexpr int T = 1 << L;
    static constexpr int NP = npasses(L);
    static constexpr int Q = T / kPow2EPT;            // threads / sequence
    static constexpr int SEQ = Q >= 256 ? 1 : 256 / Q;  // sequences / CTA
    static constexpr int THREADS = Q * SEQ;
    static constexpr int SMEM_SEQ = T + T / 32;         // padded elements
    static constexpr int TAB = tab_off(L, NP);          // float4 entries
    // two ping-pong buffers per sequence, the twiddle table, the per-sequence
    // power
    static constexpr size_t SMEM = (size_t)SEQ * 2 * SMEM_SEQ * sizeof(float2) +
                                   (size_t)TAB * sizeof(float4) +
                                   (size_t)SEQ * sizeof(float);
    // resident CTAs per SM the register budget is sized for
    static constexpr int MIN_BLOCKS = 65536 / (kPow2Regs * THREADS) > 0
                                          ? 65536 / (kPow2Regs * THREADS) : 1;
    // the last forward pass fuses with the first inverse pass
    static constexpr bool FUSED = NP >= 2 && radix_of(L, NP - 1) == kPow2EPT;
};

template <int L, int P, int NP>
__device__ __forceinline__ void fill_twiddles(float4 *tab, const float2 *__restrict__ tw) {
    if constexpr (P < NP) {
        constexpr int T = 1 << L, R = radix_of(L, P), NS = ns_of(L, P);
        constexpr int step = T / (NS * R), n = tab_len(L, P), off = tab_off(L, P);
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int sidx = i / NS, k = i & (NS - 1);
            const int ts = k * step;  // (2 sidx + 1) ts < R NS step = T
            const float2 a = __ldg(&tw[2 * sidx * ts]), b = __ldg(&tw[(2 * sidx + 1) * ts]);
            tab[off + i] = make_float4(a.x, a.y, b.x, b.y);
        }
        fill_twiddles<L, P + 1, NP>(tab, tw);
    }
}

// Pass P's inputs of this thread (B = 16/R butterflies at j = lt + q Q) from
// shared buffer src, twiddled: a[q][r] = src[j + r T/R] w^(r ts).
template <int L, int P>
__device__ __forceinline__ void pass_load(const float2 *src, const float4 *tab, int lt,
                                          float2 (&a)[kPow2EPT / radix_of(L, P)][radix_of(L, P)]) {
    constexpr int T = 1 << L, R = radix_of(L, P), NS = ns_of(L, P), B = kPow2EPT / R;
    constexpr int Q = T / kPow2EPT;
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int j = lt + q * Q;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = j + r * (T / R);
            a[q][r] = PLV_IN_BOUNDS(m < T) ? src[padi(m)] : make_float2(0.f, 0.f);
        }
        if constexpr (NS > 1) {
            const float4 *t = tab + tab_off(L, P) + (j & (NS - 1));
#pragma unroll
            for (int s2 = 0; s2 < R / 2; ++s2) {
                const float4 v = PLV_IN_BOUNDS((j & (NS - 1)) + s2 * NS < tab_len(L, P))
                                     ? t[s2 * NS] : make_float4(0.f, 0.f, 0.f, 0.f);
                if (s2 > 0) a[q][2 * s2] = cmul(a[q][2 * s2], make_float2(v.x, v.y));
                a[q][2 * s2 + 1] = cmul(a[q][2 * s2 + 1], make_float2(v.z, v.w));
            }
        }
    }
}

// Pass P's outputs: element base + r NS, base = (j - k) R + k, k = j mod NS.
template <int L, int P>
__device__ __forceinline__ void pass_store(float2 *dst, int lt,
                                           const float2 (&a)[kPow2EPT / radix_of(L, P)][radix_of(L, P)]) {
    constexpr int T = 1 << L, R = radix_of(L, P), NS = ns_of(L, P), B = kPow2EPT / R;
    constexpr int Q = T / kPow2EPT;
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int j = lt + q * Q;
        const int k = j & (NS - 1);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (PLV_IN_BOUNDS(base + r * NS < T)) dst[padi(base + r * NS)] = a[q][r];
    }
}

// The analytic mask with the inverse's 1/T, on output element m:
// conj(-i sgn(m) C) / T = sgn(m) (Im C, Re C) / T.
template <int T>
__device__ __forceinline__ float2 hilbert_mask(float2 c, int m) {
    constexpr float invT = 1.0f / (float)T;
    const float sg = (m == 0 || m == T / 2) ? 0.f : (m < T / 2 ? invT : -invT);
    return make_float2(sg * c.y, sg * c.x);
}

// A smem-to-smem pass; MASK applies the analytic mask to its outputs (the
// last forward pass when it is not fused).
template <int L, int P, bool MASK = false>
__device__ __forceinline__ void pass_smem(const float2 *src, float2 *dst, const float4 *tab,
                                          int lt) {
    constexpr int R = radix_of(L, P), B = kPow2EPT / R, NS = ns_of(L, P);
    float2 a[B][R];
    pass_load<L, P>(src, tab, lt, a);
#pragma unroll
    for (int q = 0; q < B; ++q) {
        Dft<R>::run(a[q]);
        if constexpr (MASK) {
            constexpr int Q = (1 << L) / kPow2EPT;
            const int j = lt + q * Q, k = j & (NS - 1), base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) a[q][r] = hilbert_mask<(1 << L)>(a[q][r], base + r * NS);
        }
    }
    pass_store<L, P>(dst, lt, a);
    __syncthreads();
}

// Passes P .. PEND-1 between the two buffers: pass P reads buf[P & 1].
template <int L, int P, int PEND>
__device__ __forceinline__ void passes(float2 *const (&buf)[2], const float4 *tab, int lt) {
    if constexpr (P < PEND) {
        pass_smem<L, P>(buf[P & 1], buf[(P & 1) ^ 1], tab, lt);
        passes<L, P + 1, PEND>(buf, tab, lt);
    }
}

// Optional task trait: the task's load() computes on the values it reads
// (kLoadComputes), so loading a pair early would stall the thread on those
// loads in the middle of the previous pair's passes; such tasks load at pass 0.
template <class Task, class = void>
struct LoadsEarly {
    static constexpr bool value = true;
};
template <class Task>
struct LoadsEarly<Task, decltype((void)Task::kLoadComputes)> {
    static constexpr bool value = !Task::kLoadComputes;
};

// Optional task hook: issue an L2 prefetch of the inputs of rows (r0, r1).
template <class Task, class = void>
struct HasPrefetch {
    static constexpr bool value = false;
};
template <class Task>
struct HasPrefetch<Task, decltype((void)Task::kPrefetch)> {
    static constexpr bool value = Task::kPrefetch;
};

// Bulk prefetch of `bytes` at p into L2 (a hint: skipped unless p and bytes
// are multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    if (p == nullptr || ((uintptr_t)p & 15) != 0 || (bytes & 15) != 0 || bytes == 0) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The Hilbert transform of real rows, two rows per complex FFT, for any
// Task providing
//   Rows rows(int64_t r0, bool v0, int64_t r1, bool v1):
//       per-pair state (row addresses), computed once per pair;
//   float2 load(const Rows &, int m):
//       the complex sample c[m] = u0[m] + i u1[m] of rows r0, r1;
//   void finish(const Rows &, int m, float h0, float h1, float floor2):
//       consumes H{u0}[m], H{u1}[m]; floor2 is 2^-40 of the pair's mean
//       |c|^2 (the rounding floor of the transform);
// and optionally finish8 (eight consecutive samples) and prefetch(r0, v0,
// r1, v1) (an L2 prefetch of a later pair's inputs).
template <int L, class Task>
__global__ void __launch_bounds__(K1Cfg<L>::THREADS, K1Cfg<L>::MIN_BLOCKS)
k_hilbert_pairs(const Task task, const float2 *__restrict__ tw, int64_t rows,
                int64_t nbatch) {
    using C = K1Cfg<L>;
    constexpr int T = C::T;
    constexpr int NP = C::NP;
    extern __shared__ __align__(16) float2 smem[];
    const int lt = threadIdx.x % C::Q;
    const int sq = threadIdx.x / C::Q;
    float2 *const buf[2] = {smem + (2 * sq) * C::SMEM_SEQ, smem + (2 * sq + 1) * C::SMEM_SEQ};
    float4 *const tab = reinterpret_cast<float4 *>(smem + 2 * C::SEQ * C::SMEM_SEQ);
    float *const s_pow = reinterpret_cast<float *>(tab + C::TAB);
    fill_twiddles<L, 1, NP>(tab, tw);  // ordered before use by the loop's first barriers

    // Pass 0's inputs come from registers loaded one pair ahead: the loads of
    // the next pair are issued after the fused middle pass, so their latency
    // hides behind the inverse passes and the finish (tasks whose load()
    // computes on what it reads load at pass 0 instead).
    constexpr bool EARLY = LoadsEarly<Task>::value;
    constexpr int R0 = radix_of(L, 0), B0 = kPow2EPT / R0;
    float2 xin[B0][R0];
    auto load_inputs = [&](int64_t bb) {
        const int64_t p = bb * C::SEQ + sq;
        const auto r = task.rows(2 * p, 2 * p < rows, 2 * p + 1, 2 * p + 1 < rows);
#pragma unroll
        for (int q = 0; q < B0; ++q)
#pragma unroll
            for (int k = 0; k < R0; ++k) {
                const int m = lt + q * C::Q + k * (T / R0);
                xin[q][k] = PLV_IN_BOUNDS(m < T) ? task.load(r, m) : make_float2(0.f, 0.f);
            }
    };
    if (EARLY && blockIdx.x < nbatch) load_inputs(blockIdx.x);

    for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x) {
        const int64_t pair = b * C::SEQ + sq;
        const int64_t r0 = 2 * pair, r1 = 2 * pair + 1;
        const bool v0 = r0 < rows, v1 = r1 < rows;
        if constexpr (HasPrefetch<Task>::value) {
            // L2 prefetch of the inputs two of this CTA's pairs ahead (the
            // register loads take the next one)
            if (lt == 0 && b + 2 * (int64_t)gridDim.x < nbatch) {
                const int64_t nr0 = 2 * (pair + 2 * (int64_t)gridDim.x * C::SEQ);
                task.prefetch(nr0, nr0 < rows, nr0 + 1, nr0 + 1 < rows);
            }
        }
        // the previous pair's finish is done with the buffers and s_pow
        __syncthreads();
        if (lt == 0) s_pow[sq] = 0.f;  // ordered before the adds by pass 0's barrier
        const auto rs = task.rows(r0, v0, r1, v1);
        if (!EARLY) load_inputs(b);
        // forward pass 0 from the rows, summing |c|^2
        {
            float pw = 0.f;
#pragma unroll
            for (int q = 0; q < B0; ++q) {
#pragma unroll
                for (int k = 0; k < R0; ++k)
                    pw = fmaf(xin[q][k].x, xin[q][k].x, fmaf(xin[q][k].y, xin[q][k].y, pw));
                Dft<R0>::run(xin[q]);
            }
            pass_store<L, 0>(buf[1], lt, xin);
            __syncthreads();
            // sum of |c|^2 over the sequence (its lanes are an aligned group
            // of Q threads, or whole warps when Q >= 32)
#pragma unroll
            for (int off = 1; off < (C::Q < 32 ? C::Q : 32); off <<= 1)
                pw += __shfl_xor_sync(0xffffffffu, pw, off);
            if ((lt & 31) == 0) atomicAdd(&s_pow[sq], pw);
        }
        passes<L, 1, NP - 1>(buf, tab, lt);
        // the spectrum's last forward pass, the mask and the first inverse
        // pass; FB is the buffer the first inverse pass leaves its output in
        constexpr int FB = ((NP - 1) & 1) ^ 1;
        if constexpr (C::FUSED) {
            float2 a[1][kPow2EPT];
            pass_load<L, NP - 1>(buf[(NP - 1) & 1], tab, lt, a);
            Dft<kPow2EPT>::run(a[0]);
            // element m = lt + r T/16: m < T/2 for r < 8; m = 0, T/2 at lt = 0
            constexpr float invT = 1.0f / (float)T;
#pragma unroll
            for (int r = 0; r < kPow2EPT; ++r) {
                const float sg = (lt == 0 && (r & 7) == 0) ? 0.f : (r < 8 ? invT : -invT);
                a[0][r] = make_float2(sg * a[0][r].y, sg * a[0][r].x);
            }
            Dft<kPow2EPT>::run(a[0]);
            pass_store<L, 0>(buf[FB], lt, a);
            __syncthreads();
        } else {
            pass_smem<L, NP - 1, true>(buf[(NP - 1) & 1], buf[FB], tab, lt);
            pass_smem<L, 0>(buf[FB], buf[FB ^ 1], tab, lt);
        }
        // the next pair's inputs, in flight during the inverse passes
        if (EARLY && b + gridDim.x < nbatch) load_inputs(b + gridDim.x);
        // inverse passes 1 .. NP-1: inverse pass 0 left its output in buf[O],
        // and pass p reads pbuf[p & 1]
        constexpr int O = C::FUSED ? FB : FB ^ 1;
        float2 *const pbuf[2] = {buf[O ^ 1], buf[O]};
        passes<L, 1, NP>(pbuf, tab, lt);
        const float2 *w_out = pbuf[NP & 1];

        const float floor2 = 0x1p-40f * (s_pow[sq] * (1.0f / (float)T));
        if constexpr (HasFinish8<Task>::value) {
            // eight consecutive samples per call (vector loads and stores)
#pragma unroll
            for (int u = 0; u < kPow2EPT / 8; ++u) {
                const int m0 = 8 * (lt + u * C::Q);
                float h0[8], h1[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float2 w = w_out[padi(m0 + k)];
                    h0[k] = w.x;
                    h1[k] = -w.y;
                }
                if (PLV_IN_BOUNDS(m0 + 8 <= T)) task.finish8(rs, m0, h0, h1, floor2);
            }
        } else {
#pragma unroll 4
            for (int u = 0; u < kPow2EPT; ++u) {
                const int m = lt + u * C::Q;
                const float2 w = w_out[padi(m)];
                if (PLV_IN_BOUNDS(m < T)) task.finish(rs, m, w.x, -w.y, floor2);
            }
        }
    }
}

template <int L, class Task>
cudaError_t launch_hilbert_pairs(int num_sms, cudaStream_t st, const Task &task,
                                 const float2 *tw, int64_t rows) {
    using C = K1Cfg<L>;
    auto kern = k_hilbert_pairs<L, Task>;
    static LaunchSetup ls;
    int per_sm = 0;
    cudaError_t e = setup_once(ls, kern, C::THREADS, C::SMEM, per_sm);
    if (e != cudaSuccess) return e;
    const int64_t pairs = (rows + 1) / 2;
    const int64_t nbatch = (pairs + C::SEQ - 1) / C::SEQ;
    if (nbatch == 0) return cudaSuccess;
    // one wave of persistent CTAs (each fills its twiddle table once)
    int64_t grid = (int64_t)per_sm * num_sms;
    if (grid > nbatch) grid = nbatch;
    kern<<<(unsigned)grid, C::THREADS, C::SMEM, st>>>(task, tw, rows, nbatch);
    return cudaGetLastError();
}

// Dispatch on log2(T) to the compiled lengths.
template <class Task>
cudaError_t launch_hilbert_pow2(int num_sms, cudaStream_t st, int log2T, const Task &task,
                                const float2 *tw, int64_t rows) {
    switch (log2T) {
        case 5: return launch_hilbert_pairs<5>(num_sms, st, task, tw, rows);
        case 6: return launch_hilbert_pairs<6>(num_sms, st, task, tw, rows);
        case 7: return launch_hilbert_pairs<7>(num_sms, st, task, tw, rows);
        case 8: return launch_hilbert_pairs<8>(num_sms, st, task, tw, rows);
        case 9: return launch_hilbert_pairs<9>(num_sms, st, task, tw, rows);
        case 10: return launch_hilbert_pairs<10>(num_sms, st, task, tw, rows);
        case 11: return launch_hilbert_pairs<11>(num_sms, st, task, tw, rows);
        case 12: return launch_hilbert_pairs<12>(num_sms, st, task, tw, rows);
        case 13: return launch_hilbert_pairs<13>(num_sms, st, task, tw, rows);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Any-length engine.  The periodic Hilbert transform of length T is the
// circular convolution y = x (*)_T k_T with the real, odd kernel
//     k_T[n] = (2/T) sum_{k=1}^{ceil(T/2)-1} sin(2 pi k n / T)
// (the inverse DFT of -i sgn).  A circular convolution of length T equals
// the first T outputs of a circular convolution of length M >= 2T - 1 of the
// zero-padded row with the kernel placed at [0, T) and its periodic
// continuation at [M - T + 1, M).  So for any T:
//     y = IFFT_M( K (.) FFT_M(c_pad) ),  K = FFT_M(k_circ) = -i S  (S real).
// FFT_M is an in-place decimation-in-frequency transform (digit-reversed
// output), K is stored in that order (and divided by M), and the inverse is
// the matching in-place decimation-in-time transform (digit-reversed input,
// natural output), so no reordering pass is needed.  M = 2^a, 3 * 2^a or
// 5 * 2^a.
// One sequence (row pair) per CTA; every thread loops over butterflies with
// only R values in registers, so the shared buffer is single.

__device__ __forceinline__ void dft3(float2 (&a)[3]) {
    const float h = 0.86602540378443864676f;  // sqrt(3) / 2
    const float2 t1 = cadd(a[1], a[2]);
    const float2 t2 = make_float2(fmaf(-0.5f, t1.x, a[0].x), fmaf(-0.5f, t1.y, a[0].y));
    const float2 d = csub(a[1], a[2]);
    const float2 t3 = make_float2(h * d.y, -h * d.x);  // -i h (a1 - a2)
    a[0] = cadd(a[0], t1);
    a[1] = cadd(t2, t3);
    a[2] = csub(t2, t3);
}

// Forward DFT of length 5 with w = exp(-2 pi i / 5): with t1 = a1 + a4,
// t2 = a2 + a3, t3 = a1 - a4, t4 = a2 - a3,
//   X1,4 = a0 + c1 t1 + c2 t2 -/+ i (s1 t3 + s2 t4),
//   X2,3 = a0 + c2 t1 + c1 t2 -/+ i (s2 t3 - s1 t4),
// c_k = cos(2 pi k / 5), s_k = sin(2 pi k / 5).
__device__ __forceinline__ void dft5(float2 (&a)[5]) {
    const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
    const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
    const float2 t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
    const float2 t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
    const float2 b1 = make_float2(fmaf(c2, t2.x, fmaf(c1, t1.x, a[0].x)),
                                  fmaf(c2, t2.y, fmaf(c1, t1.y, a[0].y)));
    const float2 b2 = make_float2(fmaf(c1, t2.x, fmaf(c2, t1.x, a[0].x)),
                                  fmaf(c1, t2.y, fmaf(c2, t1.y, a[0].y)));
    const float2 d1 = make_float2(fmaf(s2, t4.x, s1 * t3.x), fmaf(s2, t4.y, s1 * t3.y));
    const float2 d2 = make_float2(fmaf(-s1, t4.x, s2 * t3.x), fmaf(-s1, t4.y, s2 * t3.y));
    a[0] = cadd(a[0], cadd(t1, t2));
    // -i d = (d.y, -d.x)
    a[1] = make_float2(b1.x + d1.y, b1.y - d1.x);
    a[4] = make_float2(b1.x - d1.y, b1.y + d1.x);
    a[2] = make_float2(b2.x + d2.y, b2.y - d2.x);
    a[3] = make_float2(b2.x - d2.y, b2.y + d2.x);
}

template <int R>
__device__ __forceinline__ void dft_any(float2 (&a)[R]) {
    if constexpr (R == 3) dft3(a);
    else if constexpr (R == 5) dft5(a);
    else Dft<R>::run(a);
}

// Load R values (stride sub) of one butterfly; with INV conjugate them.
template <int R, bool INV>
__device__ __forceinline__ void bfly_load(const float2 *s, int base, int sub, float2 (&a)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        a[r] = s[padi(base + r * sub)];
        if (INV) a[r].y = -a[r].y;
    }
}
// Stage kinds of the any-length transform.
enum ConvStage { kDifSmem = 0, kDitSmem = 1, kDifFirst = 2, kMidFused = 3, kDitLast = 4 };

// The R - 1 twiddles w[r] = tw[r tb] of one butterfly position (w[0] = 1).
template <int R>
__device__ __forceinline__ void load_twiddles(float2 (&w)[R], int tb,
                                              const float2 *__restrict__ tw) {
    w[0] = make_float2(1.f, 0.f);
#pragma unroll
    for (int r = 1; r < R; ++r) w[r] = __ldg(&tw[r * tb]);
}
template <int R>
__device__ __forceinline__ void apply_twiddles(float2 (&a)[R], const float2 (&w)[R]) {
#pragma unroll
    for (int r = 1; r < R; ++r) a[r] = cmul(a[r], w[r]);
}
template <int R>
__device__ __forceinline__ void apply_twiddles_mem(float2 (&a)[R], int tb,
                                                  const float2 *__restrict__ tw) {
#pragma unroll
    for (int r = 1; r < R; ++r) a[r] = cmul(a[r], __ldg(&tw[r * tb]));
}

// One butterfly of a stage: base = g span + j, twiddles w of position j.
//   kDifFirst: inputs c[m] = task.load (0 for m >= T) straight from global
//              memory, sums |c|^2 into *pw;
//   kDifSmem / kDitSmem: shared memory in place;
//   kMidFused: the last forward stage, the multiply by K = -i S / M and the
//              first inverse stage, all in registers (same butterflies, sub = 1,
//              so j = 0 and no twiddles);
//   kDitLast:  the last inverse stage; outputs m < T go to task.finish, the
//              padding T <= m < ld to task.pad.
template <int R, int KIND, bool HOIST, class Task>
__device__ __forceinline__ void conv_butterfly(float2 *s, int base, int sub, int tb,
                                               const float2 (&w)[R], const ConvPlan &plan,
                                               const Task &task,
                                               const typename Task::Rows &rs, int T,
                                               int64_t ld, float *pw, float floor2) {
    // every value of the butterfly lies inside the transform
    if (!PLV_IN_BOUNDS(base >= 0 && base + (R - 1) * sub < plan.M)) return;
    float2 a[R];
    if constexpr (KIND == kDifFirst) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = base + r * sub;
            a[r] = m < T ? task.load(rs, m) : make_float2(0.f, 0.f);
            *pw = fmaf(a[r].x, a[r].x, fmaf(a[r].y, a[r].y, *pw));
        }
        dft_any<R>(a);
        if constexpr (HOIST) apply_twiddles<R>(a, w);
        else if (tb != 0) apply_twiddles_mem<R>(a, tb, plan.tw);
    } else if constexpr (KIND == kDifSmem) {
        bfly_load<R, false>(s, base, sub, a);
        dft_any<R>(a);
        if constexpr (HOIST) apply_twiddles<R>(a, w);
        else if (tb != 0) apply_twiddles_mem<R>(a, tb, plan.tw);
    } else if constexpr (KIND == kMidFused) {
        bfly_load<R, false>(s, base, sub, a);
        dft_any<R>(a);
        // times -i S, then conjugate for the inverse: conj(-i S v) = (S y, S x)
        float S[R];
        if constexpr (R % 4 == 0) {
            // base = g R: 16-byte aligned runs of four
#pragma unroll
            for (int q = 0; q < R; q += 4) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(plan.S + base + q));
                S[q] = v.x;
                S[q + 1] = v.y;
                S[q + 2] = v.z;
                S[q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) S[q] = __ldg(&plan.S[base + q * sub]);
        }
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = make_float2(S[q] * a[q].y, S[q] * a[q].x);
        dft_any<R>(a);
    } else {  // kDitSmem, kDitLast
        bfly_load<R, true>(s, base, sub, a);
        if constexpr (HOIST) apply_twiddles<R>(a, w);
        else if (tb != 0) apply_twiddles_mem<R>(a, tb, plan.tw);
        dft_any<R>(a);
    }
    if constexpr (KIND == kDitLast) {
        // (staging these outputs in shared memory for runs of eight vector
        // stores, as the power-of-two engine does, measured 6 % slower here)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int m = base + q * sub;
            if (m < T) task.finish(rs, m, a[q].x, -a[q].y, floor2);
            else if (m < ld) task.pad(rs, m);
        }
    } else {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            float2 v = a[q];
            if (KIND == kDitSmem || KIND == kMidFused) v.y = -v.y;
            if (PLV_IN_BOUNDS(base + q * sub < plan.M)) s[padi(base + q * sub)] = v;
        }
    }
}

// One stage over all butterflies.  span = R sub with sub = 1 << lsub;
// butterfly b is (g, j) = (b >> lsub, b & (sub - 1)), twiddle step
// tb = (M / span) j.  When sub <= blockDim (both powers of two), j is the
// same for every butterfly of a thread, so its twiddles are loaded once.
template <int R, int KIND, class Task>
__device__ __forceinline__ void conv_stage_r(float2 *s, int M, int lsub, const ConvPlan &plan,
                                             const Task &task, const typename Task::Rows &rs,
                                             int T, int64_t ld, float *pw, float floor2) {
    const int sub = 1 << lsub;
    const int span = R * sub;
    const int tstep = M / span;  // w_span = w_M^tstep
    const int nb = M / R;
    if (KIND == kMidFused || sub <= (int)blockDim.x) {
        const int tb = KIND == kMidFused ? 0 : tstep * ((int)threadIdx.x & (sub - 1));
        float2 w[R];
        if (KIND != kMidFused) load_twiddles<R>(w, tb, plan.tw);
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int g = b >> lsub, j = b & (sub - 1);
            conv_butterfly<R, KIND, KIND != kMidFused>(s, g * span + j, sub, tb, w, plan, task,
                                                       rs, T, ld, pw, floor2);
        }
    } else {
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int g = b >> lsub, j = b & (sub - 1);
            const int tb = tstep * j;
            float2 w[R];  // not read: twiddles come from memory per butterfly
            conv_butterfly<R, KIND, false>(s, g * span + j, sub, tb, w, plan, task, rs, T, ld,
                                           pw, floor2);
        }
    }
}

template <int KIND, class Task>
__device__ __forceinline__ void conv_stage(float2 *s, int M, int R, int lsub,
                                           const ConvPlan &plan, const Task &task,
                                           const typename Task::Rows &rs, int T, int64_t ld,
                                           float *pw, float floor2) {
    // radices above kConvMaxRadix never occur (the plan's schedule) and are
    // not compiled, so they do not count against the register budget
    switch (R) {
        case 16:
            if constexpr (kConvMaxRadix >= 16)
                conv_stage_r<16, KIND>(s, M, lsub, plan, task, rs, T, ld, pw, floor2);
            break;
        case 8: conv_stage_r<8, KIND>(s, M, lsub, plan, task, rs, T, ld, pw, floor2); break;
        case 5: conv_stage_r<5, KIND>(s, M, lsub, plan, task, rs, T, ld, pw, floor2); break;
        case 4: conv_stage_r<4, KIND>(s, M, lsub, plan, task, rs, T, ld, pw, floor2); break;
        case 3: conv_stage_r<3, KIND>(s, M, lsub, plan, task, rs, T, ld, pw, floor2); break;
        default: conv_stage_r<2, KIND>(s, M, lsub, plan, task, rs, T, ld, pw, floor2); break;
    }
}

__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }


// One row pair (rows 2 pr, 2 pr + 1 of `rows`) through the any-length
// engine.  Same Task interface as k_hilbert_pairs, plus
//   void pad(const Rows &, int m)
// for the padding samples T <= m < ld of the output rows.  Stages: the first
// forward stage reads global memory, the last forward and first inverse
// stages run fused in registers, the last inverse stage writes the outputs.
// Entry and exit: *s_pow is 0; the caller's threads all take part.
template <class Task>
__device__ __forceinline__ void conv_pair(const Task &task, const ConvPlan &plan, int T,
                                          int64_t ld, int64_t rows, int64_t pr, float2 *smem,
                                          float *s_pow) {
    const int M = plan.M;
    const int ns = plan.nstages;
    const int64_t r0 = 2 * pr, r1 = 2 * pr + 1;
    const bool v0 = r0 < rows, v1 = r1 < rows;
    __syncthreads();  // the previous pair is done with smem; s_pow is 0
    const auto rs = task.rows(r0, v0, r1, v1);
    // forward stages; span of stage st is M / (radix[0] ... radix[st-1])
    int span = M;
    float pw = 0.f, floor2 = 0.f;
    for (int st = 0; st < ns - 1; ++st) {
        const int R = plan.radix[st];
        const int lsub = ilog2(span / R);
        if (st == 0)
            conv_stage<kDifFirst>(smem, M, R, lsub, plan, task, rs, T, ld, &pw, 0.f);
        else
            conv_stage<kDifSmem>(smem, M, R, lsub, plan, task, rs, T, ld, nullptr, 0.f);
        if (st == 0) {
#pragma unroll
            for (int off = 1; off < 32; off <<= 1)
                pw += __shfl_xor_sync(0xffffffffu, pw, off);
            if ((threadIdx.x & 31) == 0) atomicAdd(s_pow, pw);
        }
        __syncthreads();
        if (st == 0) floor2 = 0x1p-40f * (*s_pow / (float)T);
        span /= R;
    }
    // last forward stage (sub = 1), spectrum, first inverse stage
    conv_stage<kMidFused>(smem, M, plan.radix[ns - 1], 0, plan, task, rs, T, ld, nullptr, 0.f);
    __syncthreads();
    if (threadIdx.x == 0) *s_pow = 0.f;  // every thread has read it (before the barrier)
    // remaining inverse stages; the last writes the outputs
    span = plan.radix[ns - 1];
    for (int st = ns - 2; st >= 0; --st) {
        const int R = plan.radix[st];
        const int lsub = ilog2(span);
        if (st > 0) {
            conv_stage<kDitSmem>(smem, M, R, lsub, plan, task, rs, T, ld, nullptr, 0.f);
            __syncthreads();
        } else {
            conv_stage<kDitLast>(smem, M, R, lsub, plan, task, rs, T, ld, nullptr, floor2);
        }
        span *= R;
    }
}

// Persistent over the row pairs of one problem.
template <class Task, int THREADS>
__global__ void __launch_bounds__(THREADS, 65536 / (kConvRegs * THREADS))
k_hilbert_conv(const Task task, const ConvPlan plan, int T, int64_t ld, int64_t rows) {
    extern __shared__ __align__(16) float2 smem[];
    __shared__ float s_pow;
    const int64_t npairs = (rows + 1) / 2;
    if (threadIdx.x == 0) s_pow = 0.f;
    for (int64_t pr = blockIdx.x; pr < npairs; pr += gridDim.x)
        conv_pair(task, plan, T, ld, rows, pr, smem, &s_pow);
}

template <class Task, int C>
cudaError_t launch_hilbert_conv_t(int num_sms, cudaStream_t st, const Task &task,
                                  const ConvPlan &plan, int T, int64_t ld, int64_t rows) {
    constexpr int THREADS = conv_class_threads(C);
    auto kern = k_hilbert_conv<Task, THREADS>;
    static LaunchSetup ls;
    int per_sm = 0;
    cudaError_t e = setup_once(ls, kern, THREADS, conv_smem(conv_class_max_M(C)), per_sm);
    if (e != cudaSuccess) return e;
    const int64_t npairs = (rows + 1) / 2;
    if (npairs == 0) return cudaSuccess;
    int64_t grid = (int64_t)per_sm * num_sms;
    if (grid > npairs) grid = npairs;
    kern<<<(unsigned)grid, THREADS, conv_smem(plan.M), st>>>(task, plan, T, ld, rows);
    return cudaGetLastError();
}

template <class Task>
cudaError_t launch_hilbert_conv(int num_sms, cudaStream_t st, const Task &task,
                                const ConvPlan &plan, int T, int64_t ld, int64_t rows) {
    switch (conv_class(plan.M)) {
        case 0: return launch_hilbert_conv_t<Task, 0>(num_sms, st, task, plan, T, ld, rows);
        case 1: return launch_hilbert_conv_t<Task, 1>(num_sms, st, task, plan, T, ld, rows);
        case 2: return launch_hilbert_conv_t<Task, 2>(num_sms, st, task, plan, T, ld, rows);
        default: return launch_hilbert_conv_t<Task, 3>(num_sms, st, task, plan, T, ld, rows);
    }
}

}  // namespace fft
}  // namespace plv
