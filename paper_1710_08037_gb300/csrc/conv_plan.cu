// conv_plan.cu -- host side of the any-length Hilbert transform: choice of
// the FFT length M >= 2T - 1 (2^a, 3 * 2^a or 5 * 2^a), its radix order, and the
// spectrum of the periodic discrete Hilbert kernel, computed in FP64 with the
// same in-place decimation-in-frequency algorithm the device runs, so it
// lands in the device's output order.  Tables are cached per handle.
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "common.cuh"

namespace plv {
namespace {

typedef std::complex<double> cd;

int choose_M(int T) {
    const int need = 2 * T - 1;
    int best = 0;
    for (int p = 32; p <= kMaxConvM; p *= 2)
        for (int f : {1, 3, 5})
            if (f * p >= need && f * p <= kMaxConvM && (best == 0 || f * p < best)) best = f * p;
    return best;
}

// Radix order of the transform: 3 or 5 first for M = 3 * 2^a or 5 * 2^a
// (every later span is then a power of two), then stages of the largest
// radix R = kConvMaxRadix
// and one remainder radix 2^(a mod log2 R).  The remainder goes where it leaves the fewest twiddle loads
// on the device: a stage whose sub-block length (span / R) exceeds the CTA's
// thread count loads its R - 1 twiddles per butterfly, a later one loads
// them once per thread; the last forward stage has none.
std::vector<int> schedule(int M) {
    std::vector<int> head;
    int m = M;
    for (int f : {3, 5})
        if (m % f == 0) {
            head.push_back(f);
            m /= f;
        }
    int a = 0;
    while ((1 << a) < m) ++a;
    int lr = 0;  // log2 of the largest radix
    while ((2 << lr) <= kConvMaxRadix) ++lr;
    const int n16 = a / lr, rem = 1 << (a % lr);
    const int threads = conv_threads(M);
    std::vector<int> best;
    double best_cost = 0.0;
    for (int pos = 0; pos <= n16; ++pos) {
        std::vector<int> r = head;
        for (int k = 0; k < n16; ++k) {
            if (k == pos && rem > 1) r.push_back(rem);
            r.push_back(kConvMaxRadix);
        }
        if (pos == n16 && rem > 1) r.push_back(rem);
        double cost = 0.0;
        int span = M;
        for (size_t st = 0; st < r.size(); ++st) {
            const int sub = span / r[st];
            if (st + 1 < r.size() && sub > threads) cost += (double)(r[st] - 1) / r[st];
            span = sub;
        }
        if (best.empty() || cost < best_cost) {
            best = r;
            best_cost = cost;
        }
        if (rem == 1) break;  // no remainder to place
    }
    return best;
}

// In-place decimation-in-frequency FFT with the device's loop structure.
void host_dif(std::vector<cd> &x, int M, const std::vector<int> &radix) {
    int span = M;
    std::vector<cd> v(16), V(16);
    for (int R : radix) {
        const int sub = span / R;
        for (int b = 0; b < M / R; ++b) {
            const int g = b / sub, j = b - g * sub;
            const int base = g * span + j;
            for (int r = 0; r < R; ++r) v[r] = x[base + r * sub];
            for (int q = 0; q < R; ++q) {
                cd acc = 0.0;
                for (int r = 0; r < R; ++r)
                    acc += v[r] * std::polar(1.0, -2.0 * M_PI * (double)(r * q % R) / R);
                V[q] = acc * std::polar(1.0, -2.0 * M_PI * (double)q * j / span);
            }
            for (int q = 0; q < R; ++q) x[base + q * sub] = V[q];
        }
        span = sub;
    }
}

}  // namespace

plv_status get_conv_plan(Handle &h, int T, const ConvPlan **out) {
    auto it = h.conv.find(T);
    if (it != h.conv.end()) {
        *out = &it->second;
        return PLV_OK;
    }
    const int M = choose_M(T);
    if (M == 0 || T < 2)
        return fail(PLV_ERR_UNSUPPORTED, "T = %d: lengths up to %d are supported", T,
                    kMaxConvM / 2);
    const std::vector<int> radix = schedule(M);
    // periodic Hilbert kernel k_T[n] = (2/T) sum_{k=1}^{K} sin(2 pi k n / T),
    // K = ceil(T/2) - 1, summed in closed form
    const int K = (T + 1) / 2 - 1;
    std::vector<double> kt(T, 0.0);
    for (int n = 1; n < T; ++n) {
        const double th = 2.0 * M_PI * n / T;
        const double den = sin(th / 2.0);
        kt[n] = (2.0 / T) * sin(K * th / 2.0) * sin((K + 1) * th / 2.0) / den;
    }
    std::vector<cd> kc(M, 0.0);
    for (int m = 0; m < T; ++m) kc[m] = kt[m];
    for (int j = 1; j < T; ++j) kc[M - j] = kt[T - j];
    host_dif(kc, M, radix);
    // K = FFT(k) is imaginary: K = -i S, S = -Im K; fold in 1/M
    std::vector<float> S(M);
    for (int p = 0; p < M; ++p) S[p] = (float)(-kc[p].imag() / M);
    if (!h.conv_tw.count(M)) {
        std::vector<float2> tw(M);
        for (int m = 0; m < M; ++m) {
            const double a = 2.0 * M_PI * m / M;
            tw[m] = make_float2((float)cos(a), (float)-sin(a));
        }
        float2 *d = nullptr;
        cudaError_t e = dev_malloc(&d, sizeof(float2) * M);
        if (e != cudaSuccess) return check_alloc(e, "any-length plan: twiddles");
        e = cudaMemcpy(d, tw.data(), sizeof(float2) * M, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d);
            return check_cuda(e, "any-length plan: twiddles upload");
        }
        h.conv_tw[M] = d;
        h.workspace_used += sizeof(float2) * M;
        note_usage(h);
    }
    float *dS = nullptr;
    cudaError_t e = dev_malloc(&dS, sizeof(float) * M);
    if (e != cudaSuccess) return check_alloc(e, "any-length plan: spectrum");
    e = cudaMemcpy(dS, S.data(), sizeof(float) * M, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dS);
        return check_cuda(e, "any-length plan: spectrum upload");
    }
    h.conv_S[T] = dS;
    h.workspace_used += sizeof(float) * M;
    note_usage(h);
    ConvPlan p;
    p.M = M;
    p.nstages = (int)radix.size();
    for (int k = 0; k < 8; ++k) p.radix[k] = k < p.nstages ? radix[k] : 0;
    p.tw = h.conv_tw[M];
    p.S = dS;
    h.conv[T] = p;
    *out = &h.conv[T];
    return PLV_OK;
}

namespace {

// In-place radix-2 FFT of length n (a power of two), sign -1 (forward) or +1.
void fft_pow2(std::vector<cd> &a, int sign) {
    const int n = (int)a.size();
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (int len = 2; len <= n; len <<= 1) {
        for (int i = 0; i < n; i += len)
            for (int k = 0; k < len / 2; ++k) {
                const cd w = std::polar(1.0, sign * 2.0 * M_PI * (double)k / len);
                const cd u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

// Inverse DFT of any length T in FP64 by Bluestein's chirp-z identity:
// with kn = (k^2 + n^2 - (n - k)^2) / 2,
//   y[n] = (1/T) c[n] sum_k (Y[k] c[k]) conj(c[n - k]),  c[j] = exp(i pi j^2 / T),
// a linear convolution done with power-of-two FFTs (j^2 taken mod 2T, so the
// chirp's angle stays exact).
std::vector<cd> idft_any(const std::vector<cd> &Y) {
    const int T = (int)Y.size();
    std::vector<cd> c(T);
    for (int j = 0; j < T; ++j) {
        const long long q = ((long long)j * j) % (2LL * T);
        c[j] = std::polar(1.0, M_PI * (double)q / T);
    }
    int L = 1;
    while (L < 2 * T - 1) L <<= 1;
    std::vector<cd> a(L, 0.0), b(L, 0.0);
    for (int k = 0; k < T; ++k) a[k] = Y[k] * c[k];
    b[0] = std::conj(c[0]);
    for (int j = 1; j < T; ++j) b[j] = b[L - j] = std::conj(c[j]);
    fft_pow2(a, -1);
    fft_pow2(b, -1);
    for (int i = 0; i < L; ++i) a[i] *= b[i];
    fft_pow2(a, +1);
    std::vector<cd> y(T);
    for (int n = 0; n < T; ++n) y[n] = c[n] * a[n] / ((double)L * T);
    return y;
}

uint64_t fnv1a(const void *p, size_t n, uint64_t hsh) {
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) hsh = (hsh ^ b[i]) * 1099511628211ULL;
    return hsh;
}

}  // namespace

// The host helpers of the any-length plans under external names, so that
// CPU tests can link against them: the transform length for T, its radix
// order, and the FP64 inverse DFT of any length.
int conv_length(int T) { return choose_M(T); }
std::vector<int> conv_radix_order(int M) { return schedule(M); }
std::vector<std::complex<double>> inverse_dft_any(const std::vector<std::complex<double>> &Y) {
    return idft_any(Y);
}

plv_status get_band_plan(Handle &h, cudaStream_t s, int T, const float *masks, int nbands,
                         const ConvPlan **plan, const float2 **K) {
    plv_status st = get_conv_plan(h, T, plan);
    if (st != PLV_OK) return st;
    const int M = (*plan)->M;
    const int nb = T / 2 + 1;
    std::vector<float> hm((size_t)nbands * nb);
    cudaError_t e = cudaMemcpyAsync(hm.data(), masks, sizeof(float) * hm.size(),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return check_cuda(e, "plv_analytic_bands: read the band masks");
    uint64_t key = fnv1a(&T, sizeof T, 1469598103934665603ULL);
    key = fnv1a(&nbands, sizeof nbands, key);
    key = fnv1a(hm.data(), sizeof(float) * hm.size(), key);
    auto it = h.band_K.find(key);
    if (it != h.band_K.end()) {
        *K = it->second;
        return PLV_OK;
    }
    std::vector<int> radix((*plan)->radix, (*plan)->radix + (*plan)->nstages);
    std::vector<float2> Kf((size_t)nbands * M);
    for (int b = 0; b < nbands; ++b) {
        // spectrum h B of the band-limited analytic signal on the T-point grid:
        // h[0] = 1, h[k] = 2 for 0 < k < T/2, h[T/2] = 1 (even T), 0 above;
        // the real, even mask B given at the bins 0 .. T/2
        const float *B = hm.data() + (size_t)b * nb;
        std::vector<cd> Y(T, 0.0);
        for (int k = 0; 2 * k <= T; ++k) {
            const double hk = (k == 0 || 2 * k == T) ? 1.0 : 2.0;
            Y[k] = hk * (double)B[k];
        }
        // its kernel k_b = IDFT_T(h B); z_b = x (*)_T k_b, placed for the
        // zero-padded length-M transform as for the Hilbert kernel
        const std::vector<cd> kt = idft_any(Y);
        std::vector<cd> kc(M, 0.0);
        for (int m = 0; m < T; ++m) kc[m] = kt[m];
        for (int j = 1; j < T; ++j) kc[M - j] = kt[T - j];
        host_dif(kc, M, radix);  // the device's digit-reversed order
        for (int p = 0; p < M; ++p)
            Kf[(size_t)b * M + p] =
                make_float2((float)(kc[p].real() / M), (float)(kc[p].imag() / M));
    }
    float2 *d = nullptr;
    e = dev_malloc(&d, sizeof(float2) * Kf.size());
    if (e != cudaSuccess) return check_alloc(e, "plv_analytic_bands: band kernels");
    e = cudaMemcpy(d, Kf.data(), sizeof(float2) * Kf.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return check_cuda(e, "plv_analytic_bands: band kernels upload");
    }
    h.band_K[key] = d;
    h.workspace_used += sizeof(float2) * Kf.size();
    note_usage(h);
    *K = d;
    return PLV_OK;
}

void free_conv_plans(Handle &h) {
    for (auto &kv : h.conv_tw) cudaFree(kv.second);
    for (auto &kv : h.conv_S) cudaFree(kv.second);
    for (auto &kv : h.band_K) cudaFree(kv.second);
    h.conv_tw.clear();
    h.conv_S.clear();
    h.conv.clear();
    h.band_K.clear();
}

}  // namespace plv
