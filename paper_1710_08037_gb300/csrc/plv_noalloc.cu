// plv_noalloc.cu -- plv_backward_noalloc: the backward pass without any
// allocation, for callers that cannot call cudaMalloc (see include/plv.h).
//
// Everything the pass needs beyond the caller's inputs and outputs lives in
// file-scope device arrays of fixed size, which every GPU that loads this
// library holds until the process exits:
//   g_scratch   PLV_NOALLOC_SCRATCH_BYTES of scratch (recomputed phasors,
//               reciprocal amplitudes, S = G + G^H, Gamma);
//   g_twiddles  the FFT twiddle tables for every supported length.
// (The FP32 backward has no bounded waits, so no status word is needed.)
// Host code cannot use these names as device addresses: on each device the
// first call (with that device current) looks the addresses up with
// cudaGetSymbolAddress, checks the result, and uploads the twiddles.  Later
// calls reuse the addresses.  Every buffer region is fully written before it
// is read within one call, so nothing needs clearing between calls; calls
// that overlap on the GPU share the array and race.
#include <math.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace plv {
namespace {

constexpr size_t kTwiddleCount = ((size_t)1 << (kMaxLog2T + 1)) - ((size_t)1 << kMinLog2T);

static __device__ __align__(256) unsigned char g_scratch[PLV_NOALLOC_SCRATCH_BYTES];
static __device__ __align__(256) float2 g_twiddles[kTwiddleCount];

struct DeviceState {
    bool ready = false;
    unsigned char *scratch = nullptr;
    float2 *twiddles = nullptr;
    int num_sms = 0;
};

constexpr int kMaxDevices = 64;
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

// Set-up of the current device: symbol addresses, SM count, twiddle upload.
plv_status setup_current_device(int dev, DeviceState &st) {
    if (st.ready) return PLV_OK;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return check_cuda(e, "plv_backward_noalloc: scratch address");
    st.scratch = (unsigned char *)p;
    e = cudaGetSymbolAddress(&p, g_twiddles);
    if (e != cudaSuccess) return check_cuda(e, "plv_backward_noalloc: twiddle address");
    st.twiddles = (float2 *)p;
    e = cudaDeviceGetAttribute(&st.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return check_cuda(e, "plv_backward_noalloc: SM count");
    std::vector<float2> tw(kTwiddleCount);
    for (int L = kMinLog2T; L <= kMaxLog2T; ++L) {
        const size_t base = ((size_t)1 << L) - ((size_t)1 << kMinLog2T);
        const int T = 1 << L;
        for (int m = 0; m < T; ++m) {
            const double a = 2.0 * M_PI * (double)m / (double)T;
            tw[base + m] = make_float2((float)cos(a), (float)-sin(a));
        }
    }
    e = cudaMemcpyToSymbol(g_twiddles, tw.data(), kTwiddleCount * sizeof(float2));
    if (e != cudaSuccess) return check_cuda(e, "plv_backward_noalloc: twiddle upload");
    st.ready = true;
    return PLV_OK;
}

}  // namespace

// Scratch the no-allocation backward needs, with the same partition as
// plv_backward.
size_t noalloc_scratch_bytes(int batch, int N, int T) {
    const int64_t ld = padded_len(T);
    const size_t rows = (size_t)batch * N;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return up(rows * 2 * ld * 4) + up(rows * ld * 4) + up(rows * 2 * ld * 4) +
           up((size_t)batch * 2 * N * N * 4);
}

}  // namespace plv

using namespace plv;

extern "C" plv_status plv_backward_noalloc(void *stream, const void *x, plv_dtype dtype,
                                           int batch, int N, int T, int64_t ldx,
                                           const void *C, const float *g_plv,
                                           const float *g_iplv, const float *g_ciplv,
                                           float *grad_x) {
    if (batch < 0 || N < 0 || T <= 0)
        return fail(PLV_ERR_INVALID, "plv_backward_noalloc: bad sizes batch=%d N=%d T=%d",
                    batch, N, T);
    if (dtype != PLV_F32 && dtype != PLV_F64)
        return fail(PLV_ERR_INVALID, "plv_backward_noalloc: unknown dtype %d", (int)dtype);
    if (ldx < T) return fail(PLV_ERR_INVALID, "plv_backward_noalloc: ldx < T");
    if (batch == 0 || N == 0) return PLV_OK;
    if (!grad_x) return fail(PLV_ERR_INVALID, "plv_backward_noalloc: grad_x is NULL");
    int L = -1;
    if ((T & (T - 1)) == 0)
        for (L = 0; (1 << L) < T; ++L) {
        }
    if (L < kMinLog2T || L > kMaxLog2Direct)
        return fail(PLV_ERR_UNSUPPORTED,
                    "plv_backward_noalloc: T = %d (powers of two from %d to %d)", T,
                    1 << kMinLog2T, 1 << kMaxLog2Direct);
    const size_t need = noalloc_scratch_bytes(batch, N, T);
    if (need > (size_t)PLV_NOALLOC_SCRATCH_BYTES)
        return fail(PLV_ERR_INVALID,
                    "plv_backward_noalloc: batch=%d N=%d T=%d needs %zu bytes of scratch; "
                    "this entry point has a fixed %zu bytes (use plv_backward, which "
                    "allocates, for larger problems)",
                    batch, N, T, need, (size_t)PLV_NOALLOC_SCRATCH_BYTES);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return check_cuda(e, "plv_backward_noalloc: current device");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(PLV_ERR_UNSUPPORTED, "plv_backward_noalloc: device %d", dev);
    DeviceState *st;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        st = &g_dev[dev];
        plv_status s0 = setup_current_device(dev, *st);
        if (s0 != PLV_OK) return s0;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (!g_plv && !g_iplv && !g_ciplv)
        return check_cuda(cudaMemsetAsync(grad_x, 0, sizeof(float) * (size_t)batch * N * T, s),
                          "plv_backward_noalloc: zero grad");
    if (!x || !C) return fail(PLV_ERR_INVALID, "plv_backward_noalloc: NULL x or C");
    if (((uintptr_t)C % 8) != 0 || ((uintptr_t)x % (dtype == PLV_F32 ? 4 : 8)) != 0 ||
        ((uintptr_t)grad_x % 4) != 0)
        return fail(PLV_ERR_INVALID, "plv_backward_noalloc: misaligned pointer");

    // a handle view over the static arrays (no allocation)
    Handle h;
    h.device = dev;
    h.prec = PLV_PREC_FP32;
    h.num_sms = st->num_sms;
    h.twiddles = st->twiddles;
    h.status = nullptr;  // no kernel of the FP32 backward writes a status

    const int64_t ld = padded_len(T);
    const size_t rows = (size_t)batch * N;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t bP = up(rows * 2 * ld * 4), bR = up(rows * ld * 4), bG = up(rows * 2 * ld * 4);
    unsigned char *w = st->scratch;
    float *P = (float *)w, *rinv = (float *)(w + bP), *Gm = (float *)(w + bP + bR),
          *S = (float *)(w + bP + bR + bG);
    plv_status r = check_cuda(
        launch_bwd_prep(&h, s, x, dtype, (int64_t)rows, L, ldx, P, rinv, T, nullptr),
        "plv_backward_noalloc: recompute");
    if (r != PLV_OK) return r;
    return check_cuda(launch_backward(&h, s, batch, N, T, L, (const float2 *)C, g_plv, g_iplv,
                                      g_ciplv, P, rinv, S, Gm, grad_x, nullptr, nullptr, nullptr),
                      "plv_backward_noalloc launch");
}
