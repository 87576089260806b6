// k_bands.cu -- the band-pass and the analytic signal in one transform, for
// several bands at once (the band-pass then analytic signal of Section III.A,
// Eq. 3), fused with the unit phasors (Eq. 4): one forward FFT per row pair,
// then per band two inverse FFTs and the phasor store.
//
// With c = x0 + i x1 (two real rows) and a real band mask B (B[k] = B[-k]):
//   IFFT(B C)            = u0 + i u1         (u = the band-passed rows),
//   IFFT(-i sgn(k) B C)  = H{u0} + i H{u1},
// so both rows' analytic signals z_r = u_r + i H{u_r} come from two inverse
// transforms, each done as a conjugated forward FFT.  The spectrum C stays
// in a third shared buffer for all bands.  Compiled like k_fwd.cu, once per
// (input type, operand precision): -DPLV_K1_F64, -DPLV_K1_KIND (the backward
// kind compiles nothing).  Lengths: T = 2^L, L = kMinLog2Bands .. 13.
#include "analytic.cuh"

#if !defined(PLV_K1_F64) || !defined(PLV_K1_KIND)
#error "k_bands.cu is compiled with -DPLV_K1_F64=... -DPLV_K1_KIND=..."
#endif

namespace plv {

#if PLV_K1_KIND != 3

namespace {

using namespace fft;

template <int L>
struct BandCfg {
    using C = K1Cfg<L>;
    // three buffers per sequence (forward spectrum, two ping-pong), power
    static constexpr size_t SMEM =
        (size_t)C::SEQ * 3 * C::SMEM_SEQ * sizeof(float2) + (size_t)C::SEQ * sizeof(float);
};

// The first inverse pass reads the kept spectrum C from shared memory and
// applies mask and conjugation: conj(B C) = B (Re C, -Im C) for the band-
// passed pair; conj(-i sgn B C) = sgn B (Im C, Re C) for its Hilbert pair.
template <int T, bool HILBERT>
struct SpecLoad {
    const float2 *S;
    const float *band;  // floor(T/2) + 1 values
    __device__ float2 operator()(int m) const {
        const float2 c = S[padi(m)];
        const float b = __ldg(&band[m <= T / 2 ? m : T - m]);
        if (HILBERT) {
            const float sg = (m == 0 || m == T / 2) ? 0.f : (m < T / 2 ? 1.f : -1.f);
            return make_float2(sg * b * c.y, sg * b * c.x);
        }
        return make_float2(b * c.x, -b * c.y);
    }
};

template <int L, typename Tin, int PREC>
__global__ void __launch_bounds__(K1Cfg<L>::THREADS, K1Cfg<L>::MIN_BLOCKS)
k_hilbert_bands(const Tin *__restrict__ x, int64_t ldx, int N, int64_t rows, int64_t nbatch,
                const float *__restrict__ masks, int nbands, uint8_t *P, int64_t band_bytes,
                const float2 *__restrict__ tw) {
    using C = K1Cfg<L>;
    constexpr int T = C::T;
    constexpr int NP = npasses(L);
    constexpr int64_t ld = T;
    constexpr int NCH = kPow2EPT / 8;  // runs of eight samples per thread
    extern __shared__ __align__(16) float2 smem[];
    const int lt = threadIdx.x % C::Q;
    const int sq = threadIdx.x / C::Q;
    float2 *const S = smem + (3 * sq) * C::SMEM_SEQ;
    float2 *const buf[2] = {smem + (3 * sq + 1) * C::SMEM_SEQ, smem + (3 * sq + 2) * C::SMEM_SEQ};
    float *s_pow = (float *)(smem + 3 * C::SEQ * C::SMEM_SEQ);
    constexpr float invT = 1.0f / (float)T;
    const float2 *out_buf = buf[((NP - 1) & 1) ^ 1];  // where a transform ends

    for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
        const int64_t pair = bt * C::SEQ + sq;
        const int64_t r0 = 2 * pair, r1 = 2 * pair + 1;
        const bool v0 = r0 < rows, v1 = r1 < rows;
        const Tin *x0 = v0 ? x + r0 * ldx : nullptr;
        const Tin *x1 = v1 ? x + r1 * ldx : nullptr;
        const RowAddr<PREC> a0 = row_addr<PREC>(v0 ? r0 : 0, N, ld);
        const RowAddr<PREC> a1 = row_addr<PREC>(v1 ? r1 : 0, N, ld);
        __syncthreads();  // the previous pair is done with the buffers
        // forward FFT of c = x0 + i x1 into S (natural order)
        float pw;
        auto load_x = [&](int m) {
            return make_float2(x0 ? ldx_f(x0 + m) : 0.f, x1 ? ldx_f(x1 + m) : 0.f);
        };
        stockham<T, radix_of(L, 0), 1, kFromX>(nullptr, buf[1], tw, lt, load_x, &pw);
        middle_passes<L, 1, NP - 1>(buf, tw, lt);
        stockham<T, radix_of(L, NP - 1), ns_of(L, NP - 1), kSmem>(buf[(NP - 1) & 1], S, tw,
                                                                  lt, NoLoad{});
        for (int b = 0; b < nbands; ++b) {
            const float *band = masks + (int64_t)b * (T / 2 + 1);
            if (lt == 0) s_pow[sq] = 0.f;  // ordered before the adds by pass 0's barrier
            // band-passed pair: u0 + i u1 = conj(FFT(conj(B C))) / T
            stockham<T, radix_of(L, 0), 1, kFromX>(nullptr, buf[1], tw, lt,
                                                   SpecLoad<T, false>{S, band}, &pw);
#pragma unroll
            for (int off = 1; off < (C::Q < 32 ? C::Q : 32); off <<= 1)
                pw += __shfl_xor_sync(0xffffffffu, pw, off);
            if ((lt & 31) == 0) atomicAdd(&s_pow[sq], pw);
            middle_passes<L, 1, NP - 1>(buf, tw, lt);
            stockham<T, radix_of(L, NP - 1), ns_of(L, NP - 1), kSmem>(
                buf[(NP - 1) & 1], buf[((NP - 1) & 1) ^ 1], tw, lt, NoLoad{});
            // sum_k |B C|^2 = T sum_t |u0 + i u1|^2: the pair's mean power per
            // sample is that / T^2; |z|^2 below 2^-40 of it counts as zero
            const float floor2 = 0x1p-40f * (s_pow[sq] * invT * invT);
            float2 u[NCH][8];
#pragma unroll
            for (int c = 0; c < NCH; ++c)
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float2 w = out_buf[padi(8 * (lt + c * C::Q) + k)];
                    u[c][k] = make_float2(w.x * invT, -w.y * invT);  // (u0, u1)
                }
            __syncthreads();  // every thread holds its u before buf[1] is rewritten
            // Hilbert pair: H{u0} + i H{u1}
            float pw2;
            stockham<T, radix_of(L, 0), 1, kFromX>(nullptr, buf[1], tw, lt,
                                                   SpecLoad<T, true>{S, band}, &pw2);
            middle_passes<L, 1, NP - 1>(buf, tw, lt);
            stockham<T, radix_of(L, NP - 1), ns_of(L, NP - 1), kSmem>(
                buf[(NP - 1) & 1], buf[((NP - 1) & 1) ^ 1], tw, lt, NoLoad{});
            uint8_t *Pb = P + (int64_t)b * band_bytes;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int m0 = 8 * (lt + c * C::Q);
                float2 p0[8], p1[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float2 w = out_buf[padi(m0 + k)];
                    const float h0 = w.x * invT, h1 = -w.y * invT;
                    p0[k] = unit_phasor(u[c][k].x, h0, floor2);
                    p1[k] = unit_phasor(u[c][k].y, h1, floor2);
                }
                if (v0) store_phasor8<PREC>(Pb, a0, ld, m0, p0);
                if (v1) store_phasor8<PREC>(Pb, a1, ld, m0, p1);
            }
            __syncthreads();  // the next band rewrites buf[1] and s_pow
        }
    }
}

template <int L, typename Tin, int PREC>
cudaError_t launch_bands_l(const Handle *h, cudaStream_t st, const Tin *x, int64_t ldx, int N,
                           int64_t rows, const float *masks, int nbands, void *P,
                           int64_t band_bytes) {
    using C = K1Cfg<L>;
    auto kern = k_hilbert_bands<L, Tin, PREC>;
    static LaunchSetup ls;
    int per_sm = 0;
    cudaError_t e = setup_once(ls, kern, C::THREADS, BandCfg<L>::SMEM, per_sm);
    if (e != cudaSuccess) return e;
    const int64_t pairs = (rows + 1) / 2;
    const int64_t nbatch = (pairs + C::SEQ - 1) / C::SEQ;
    if (nbatch == 0) return cudaSuccess;
    int64_t grid = (int64_t)per_sm * h->num_sms;
    if (grid > nbatch) grid = nbatch;
    kern<<<(unsigned)grid, C::THREADS, BandCfg<L>::SMEM, st>>>(
        x, ldx, N, rows, nbatch, masks, nbands, (uint8_t *)P, band_bytes,
        twiddle_table(h, L));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Any other length T: z_b = x (*)_T k_b with the complex kernel
// k_b = IDFT_T(h B_b), by the zero-padded transform of length M of the
// any-length engine (fft.cuh).  A complex kernel mixes the real and imaginary
// parts, so each transform carries one row (c = x + 0i).  Per row: the
// forward stages, the last one writing the spectrum to the CTA's scratch
// slot; per band: spectrum times K_b (from scratch, in registers) fused with
// the first inverse stage, the inverse stages, and the last one storing the
// band's unit phasors.  The last forward stage and the first inverse stage
// have the same butterflies (R consecutive values at base = b R) on the same
// threads, so a thread only reads scratch values it wrote and smem values it
// overwrites itself: no barrier is needed between them.

// One row of x in, the unit phasors of band `band` out.
template <typename Tin, int PREC>
struct BandRowTask {
    const Tin *x;
    int64_t ldx;
    uint8_t *P;  // band 0's operand buffer; band b at P + b band_bytes
    int N;
    int64_t ld;
    int64_t band_bytes;
    int band;
    struct Rows {
        const Tin *x0;
        RowAddr<PREC> a0;
    };
    __device__ Rows rows(int64_t r0, bool, int64_t, bool) const {
        Rows rs;
        rs.x0 = x + r0 * ldx;
        rs.a0 = row_addr<PREC>(r0, N, ld);
        return rs;
    }
    __device__ float2 load(const Rows &rs, int m) const {
        return make_float2(ldx_f(rs.x0 + m), 0.f);
    }
    __device__ void finish(const Rows &rs, int m, float zr, float zi, float floor2) const {
        store_phasor<PREC>(P + band * band_bytes, rs.a0, ld, m, unit_phasor(zr, zi, floor2));
    }
    __device__ void pad(const Rows &rs, int m) const {
        store_phasor<PREC>(P + band * band_bytes, rs.a0, ld, m, make_float2(0.f, 0.f));
    }
};

// The last forward stage (sub = 1) from smem to the scratch slot.
template <int R>
__device__ __forceinline__ void last_fwd_to_scratch(const float2 *s, int M, float2 *scr) {
    for (int b = threadIdx.x; b < M / R; b += blockDim.x) {
        const int base = b * R;
        float2 a[R];
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = s[padi(base + q)];
        dft_any<R>(a);
#pragma unroll
        for (int q = 0; q < R; ++q) scr[base + q] = a[q];
    }
}

// Spectrum times K (complex), conjugated for the inverse, and the first
// inverse stage (sub = 1) into smem; the store conjugates back, as the
// engine's fused middle stage does.
template <int R>
__device__ __forceinline__ void band_first_inv(float2 *s, int M, const float2 *scr,
                                               const float2 *__restrict__ K) {
    for (int b = threadIdx.x; b < M / R; b += blockDim.x) {
        const int base = b * R;
        float2 a[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const float2 v = scr[base + q], k = __ldg(&K[base + q]);
            const float2 w = cmul(v, k);
            a[q] = make_float2(w.x, -w.y);
        }
        dft_any<R>(a);
#pragma unroll
        for (int q = 0; q < R; ++q) s[padi(base + q)] = make_float2(a[q].x, -a[q].y);
    }
}

__device__ __forceinline__ void last_fwd_to_scratch_any(const float2 *s, int M, int R,
                                                        float2 *scr) {
    switch (R) {
        case 8: last_fwd_to_scratch<8>(s, M, scr); break;
        case 5: last_fwd_to_scratch<5>(s, M, scr); break;
        case 4: last_fwd_to_scratch<4>(s, M, scr); break;
        case 3: last_fwd_to_scratch<3>(s, M, scr); break;
        default: last_fwd_to_scratch<2>(s, M, scr); break;
    }
}
__device__ __forceinline__ void band_first_inv_any(float2 *s, int M, int R, const float2 *scr,
                                                   const float2 *K) {
    switch (R) {
        case 8: band_first_inv<8>(s, M, scr, K); break;
        case 5: band_first_inv<5>(s, M, scr, K); break;
        case 4: band_first_inv<4>(s, M, scr, K); break;
        case 3: band_first_inv<3>(s, M, scr, K); break;
        default: band_first_inv<2>(s, M, scr, K); break;
    }
}

// Persistent over rows; CTA b uses scratch slot b (M complex values).
template <typename Tin, int PREC, int THREADS>
__global__ void __launch_bounds__(THREADS, 65536 / (kConvRegs * THREADS))
k_hilbert_conv_bands(const BandRowTask<Tin, PREC> task, const ConvPlan plan, int T,
                     int64_t rows, const float2 *__restrict__ K, int nbands,
                     float2 *__restrict__ scratch) {
    extern __shared__ __align__(16) float2 smem[];
    __shared__ float s_pow;
    const int M = plan.M;
    const int ns = plan.nstages;
    const int64_t ld = task.ld;
    float2 *scr = scratch + (int64_t)blockIdx.x * M;
    if (threadIdx.x == 0) s_pow = 0.f;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        __syncthreads();  // the previous row is done with smem; s_pow is 0
        const auto rs = task.rows(r, true, 0, false);
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
                if ((threadIdx.x & 31) == 0) atomicAdd(&s_pow, pw);
            }
            __syncthreads();
            // |z_b|^2 below 2^-40 of the row's mean power |x|^2 counts as 0
            if (st == 0) floor2 = 0x1p-40f * (s_pow / (float)T);
            span /= R;
        }
        const int Rl = plan.radix[ns - 1];
        last_fwd_to_scratch_any(smem, M, Rl, scr);
        for (int b = 0; b < nbands; ++b) {
            band_first_inv_any(smem, M, Rl, scr, K + (int64_t)b * M);
            __syncthreads();
            if (b == 0 && threadIdx.x == 0) s_pow = 0.f;  // every thread has read it
            BandRowTask<Tin, PREC> tb = task;
            tb.band = b;
            span = Rl;
            for (int st = ns - 2; st >= 0; --st) {
                const int R = plan.radix[st];
                const int lsub = ilog2(span);
                if (st > 0) {
                    conv_stage<kDitSmem>(smem, M, R, lsub, plan, tb, rs, T, ld, nullptr, 0.f);
                    __syncthreads();
                } else {
                    conv_stage<kDitLast>(smem, M, R, lsub, plan, tb, rs, T, ld, nullptr,
                                         floor2);
                }
                span *= R;
            }
            __syncthreads();  // the last stage's smem reads are done before the next band
        }
    }
}

template <typename Tin, int PREC, int C>
cudaError_t launch_bands_conv_c(const Handle *h, cudaStream_t st,
                                const BandRowTask<Tin, PREC> &task, const ConvPlan &plan, int T,
                                int64_t rows, const float2 *K, int nbands, float2 *scratch) {
    constexpr int THREADS = conv_class_threads(C);
    auto kern = k_hilbert_conv_bands<Tin, PREC, THREADS>;
    static LaunchSetup ls;
    int per_sm = 0;
    cudaError_t e = setup_once(ls, kern, THREADS, conv_smem(conv_class_max_M(C)), per_sm);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)per_sm * h->num_sms;
    const int64_t slots = conv_grid(h->num_sms, plan.M);  // scratch slots the caller sized
    if (grid > slots) grid = slots;
    if (grid > rows) grid = rows;
    if (grid <= 0) return cudaSuccess;
    kern<<<(unsigned)grid, THREADS, conv_smem(plan.M), st>>>(task, plan, T, rows, K, nbands,
                                                             scratch);
    return cudaGetLastError();
}

}  // namespace

template <typename Tin, int PREC>
cudaError_t launch_bands_conv(const Handle *h, cudaStream_t st, const Tin *x, int64_t ldx,
                              int N, int64_t rows, int T, const ConvPlan &plan, const float2 *K,
                              int nbands, void *P, int64_t band_bytes, float2 *scratch) {
    const BandRowTask<Tin, PREC> task{x, ldx, (uint8_t *)P, N, padded_len(T), band_bytes, 0};
    switch (conv_class(plan.M)) {
        case 0: return launch_bands_conv_c<Tin, PREC, 0>(h, st, task, plan, T, rows, K, nbands, scratch);
        case 1: return launch_bands_conv_c<Tin, PREC, 1>(h, st, task, plan, T, rows, K, nbands, scratch);
        case 2: return launch_bands_conv_c<Tin, PREC, 2>(h, st, task, plan, T, rows, K, nbands, scratch);
        default: return launch_bands_conv_c<Tin, PREC, 3>(h, st, task, plan, T, rows, K, nbands, scratch);
    }
}

template <typename Tin, int PREC>
cudaError_t launch_bands(const Handle *h, cudaStream_t st, const Tin *x, int64_t ldx, int N,
                         int64_t rows, int log2T, const float *masks, int nbands, void *P,
                         int64_t band_bytes) {
#define PLV_BANDS_CASE(LL)                                                                    \
    case LL:                                                                                 \
        return launch_bands_l<LL, Tin, PREC>(h, st, x, ldx, N, rows, masks, nbands, P,      \
                                             band_bytes);
    switch (log2T) {
        PLV_BANDS_CASE(7)
        PLV_BANDS_CASE(8)
        PLV_BANDS_CASE(9)
        PLV_BANDS_CASE(10)
        PLV_BANDS_CASE(11)
        PLV_BANDS_CASE(12)
        PLV_BANDS_CASE(13)
        default: return cudaErrorInvalidValue;
    }
#undef PLV_BANDS_CASE
}

#if PLV_K1_F64
template cudaError_t launch_bands<double, PLV_K1_KIND>(const Handle *, cudaStream_t,
                                                        const double *, int64_t, int, int64_t,
                                                        int, const float *, int, void *, int64_t);
template cudaError_t launch_bands_conv<double, PLV_K1_KIND>(
    const Handle *, cudaStream_t, const double *, int64_t, int, int64_t, int, const ConvPlan &,
    const float2 *, int, void *, int64_t, float2 *);
#else
template cudaError_t launch_bands<float, PLV_K1_KIND>(const Handle *, cudaStream_t,
                                                       const float *, int64_t, int, int64_t, int,
                                                       const float *, int, void *, int64_t);
template cudaError_t launch_bands_conv<float, PLV_K1_KIND>(
    const Handle *, cudaStream_t, const float *, int64_t, int, int64_t, int, const ConvPlan &,
    const float2 *, int, void *, int64_t, float2 *);
#endif

#endif  // PLV_K1_KIND != 3

}  // namespace plv
