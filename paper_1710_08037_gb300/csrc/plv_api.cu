// plv_api.cu -- the C ABI (include/plv.h): handle life cycle, host-side
// validation, dispatch to the kernels, status reporting.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "group.cuh"

namespace plv {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

plv_status fail(plv_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

plv_status check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return PLV_OK;
    return fail(PLV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---- checked builds: the registry of per-unit recording words -------------
static std::vector<CheckReader> &check_units() {
    static std::vector<CheckReader> v;
    return v;
}
int register_check_unit(CheckReader r) {
    check_units().push_back(r);
    return 0;
}

// ---- host-side fault injection ---------------------------------------------
static std::atomic<int> g_fault_kind{PLV_FAULT_NONE};
static std::atomic<int> g_fault_left{0};

bool take_fault(int kind) {
    if (g_fault_kind.load() != kind) return false;
    if (g_fault_left.fetch_sub(1) != 1) return false;
    g_fault_kind.store(PLV_FAULT_NONE);
    return true;
}

cudaError_t dev_malloc_raw(void **p, size_t bytes) {
    if (take_fault(PLV_FAULT_ALLOC)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

// PLV_FAULT = "alloc[:n]" | "launch[:n]" | "timeout", read at load time.
static void arm_fault_from_env() {
    const char *v = getenv("PLV_FAULT");
    if (!v || !*v) return;
    int kind = PLV_FAULT_NONE;
    const char *rest = nullptr;
    if (strncmp(v, "alloc", 5) == 0) { kind = PLV_FAULT_ALLOC; rest = v + 5; }
    else if (strncmp(v, "launch", 6) == 0) { kind = PLV_FAULT_LAUNCH; rest = v + 6; }
    else if (strcmp(v, "timeout") == 0) { kind = PLV_FAULT_STALL; rest = v + 7; }
    else return;
    int n = 1;
    if (*rest == ':') {
        char *end = nullptr;
        const long k = strtol(rest + 1, &end, 10);
        if (end == rest + 1 || *end != '\0' || k < 1 || k > 1000000) return;
        n = (int)k;
    } else if (*rest != '\0') {
        return;
    }
    g_fault_left.store(n);
    g_fault_kind.store(kind);
}
static const int g_fault_env_read = (arm_fault_from_env(), 0);

plv_status check_alloc(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return PLV_OK;
    cudaGetLastError();  // an allocation failure is not sticky
    return fail(PLV_ERR_ALLOC, "%s: %s", what, cudaGetErrorString(e));
}

static int log2_exact(int T) {
    if (T <= 0 || (T & (T - 1))) return -1;
    int l = 0;
    while ((1 << l) < T) ++l;
    return l;
}

// Grow the handle's scratch to at least `bytes`.  Growing allocates, which
// is refused while `s` is capturing a graph.  A scratch buffer that a capture
// used may be referenced by a graph the caller still replays, so growth keeps
// it (retired, still counted in the workspace) until plv_destroy; a buffer no
// capture used is freed.
static plv_status ensure_workspace(Handle &h, cudaStream_t s, size_t bytes) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing =
        cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
    if (h.ws_bytes >= bytes) {
        if (capturing) h.ws_in_graph = true;
        return PLV_OK;
    }
    if (capturing)
        return fail(PLV_ERR_INVALID,
                    "scratch must grow to %zu bytes while the stream is capturing; "
                    "make one call of the same size outside the capture first", bytes);
    const bool keep = h.ws && h.ws_in_graph;
    const size_t others = h.workspace_used - (keep ? 0 : h.ws_bytes);
    if (h.workspace_limit && others + bytes > h.workspace_limit)
        return fail(PLV_ERR_ALLOC, "scratch of %zu bytes exceeds the workspace limit %zu",
                    bytes, h.workspace_limit);
    if (h.ws) {
        if (keep) {
            h.ws_retired.push_back(h.ws);
        } else {
            cudaError_t e = cudaFree(h.ws);  // synchronises with work still using it
            if (e != cudaSuccess) {
                h.ws = nullptr;
                h.workspace_used = others;
                h.ws_bytes = 0;
                return check_cuda(e, "cudaFree(scratch)");
            }
        }
        h.ws = nullptr;
        h.ws_bytes = 0;
        h.ws_in_graph = false;
        h.workspace_used = others;
    }
    cudaError_t e = dev_malloc(&h.ws, bytes);
    if (e != cudaSuccess) {
        h.ws = nullptr;
        cudaGetLastError();
        return fail(PLV_ERR_ALLOC, "cudaMalloc(%zu) for scratch: %s", bytes,
                    cudaGetErrorString(e));
    }
    h.ws_bytes = bytes;
    h.workspace_used = others + bytes;
    note_usage(h);
    return PLV_OK;
}

}  // namespace plv

using namespace plv;

#define PLV_GUARD(hh)                                                      \
    DeviceGuard guard_((hh)->device);                                      \
    if (!guard_.ok) return fail(PLV_ERR_CUDA, "cannot select device %d",  \
                                (hh)->device)

extern "C" {

plv_status plv_create(plv_handle **out, int device, plv_precision prec,
                      size_t workspace_limit) {
    PLV_RANGE("plv_create");
    if (!out) return fail(PLV_ERR_INVALID, "plv_create: handle pointer is NULL");
    *out = nullptr;
    if (prec != PLV_PREC_FP32 && prec != PLV_PREC_BF16X3 && prec != PLV_PREC_FP16X3)
        return fail(PLV_ERR_INVALID, "plv_create: unknown precision %d", (int)prec);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(PLV_ERR_INVALID, "plv_create: no CUDA device %d", device);
    plv_handle *hp = new (std::nothrow) plv_handle();
    if (!hp) return fail(PLV_ERR_ALLOC, "plv_create: out of host memory");
    Handle &h = hp->h;
    h.device = device;
    h.prec = prec;
    h.workspace_limit = workspace_limit;
    DeviceGuard guard(device);
    if (!guard.ok) { delete hp; return fail(PLV_ERR_CUDA, "cannot select device %d", device); }
    plv_status st = check_cuda(
        cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, device),
        "cudaDeviceGetAttribute");
    // twiddle tables exp(-2 pi i m / 2^L), rounded from FP64
    size_t ntw = ((size_t)1 << (kMaxLog2T + 1)) - ((size_t)1 << kMinLog2T);
    std::vector<float2> tw(ntw);
    for (int L = kMinLog2T; L <= kMaxLog2T; ++L) {
        const size_t base = ((size_t)1 << L) - ((size_t)1 << kMinLog2T);
        const int T = 1 << L;
        for (int m = 0; m < T; ++m) {
            const double a = 2.0 * M_PI * (double)m / (double)T;
            tw[base + m] = make_float2((float)cos(a), (float)-sin(a));
        }
    }
    const size_t need = ntw * sizeof(float2) + 256;
    if (st == PLV_OK && workspace_limit && need > workspace_limit)
        st = fail(PLV_ERR_ALLOC, "plv_create: workspace limit %zu below %zu bytes",
                  workspace_limit, need);
    if (st == PLV_OK)
        st = check_alloc(dev_malloc(&h.twiddles, ntw * sizeof(float2)), "cudaMalloc(twiddles)");
    if (st == PLV_OK)
        st = check_cuda(cudaMemcpy(h.twiddles, tw.data(), ntw * sizeof(float2),
                                   cudaMemcpyHostToDevice), "cudaMemcpy(twiddles)");
    if (st == PLV_OK)
        st = check_alloc(dev_malloc(&h.status, 256), "cudaMalloc(status)");
    if (st == PLV_OK)
        st = check_cuda(cudaMemset(h.status, 0, 256), "cudaMemset(status)");
    if (st != PLV_OK) {
        if (h.twiddles) cudaFree(h.twiddles);
        if (h.status) cudaFree(h.status);
        delete hp;
        return st;
    }
    h.workspace_used = need;
    note_usage(h);
    *out = hp;
    return PLV_OK;
}

plv_status plv_destroy(plv_handle *hp) {
    PLV_RANGE("plv_destroy");
    if (!hp) return PLV_OK;
    Handle &h = hp->h;
    {
        DeviceGuard guard(h.device);
        cudaDeviceSynchronize();
        if (h.twiddles) cudaFree(h.twiddles);
        if (h.status) cudaFree(h.status);
        if (h.ws) cudaFree(h.ws);
        for (void *p : h.ws_retired) cudaFree(p);
        free_conv_plans(h);
    }
    delete hp;
    return PLV_OK;
}

const char *plv_last_error(const plv_handle *) { return g_err.c_str(); }

plv_precision plv_get_precision(const plv_handle *hp) {
    return hp ? hp->h.prec : PLV_PREC_FP32;
}

plv_status plv_set_gram_raster(plv_handle *hp, int width) {
    if (!hp) return fail(PLV_ERR_INVALID, "plv_set_gram_raster: NULL handle");
    if (width < 0) return fail(PLV_ERR_INVALID, "plv_set_gram_raster: width %d < 0", width);
    hp->h.gram_raster = width == 0 ? kDefaultRaster : width;
    return PLV_OK;
}

plv_status plv_set_wait_limit(plv_handle *hp, uint64_t ns) {
    if (!hp) return fail(PLV_ERR_INVALID, "plv_set_wait_limit: NULL handle");
    hp->h.wait_ns = ns == 0 ? kDefaultWaitNs : ns;
    return PLV_OK;
}

plv_status plv_check_status(plv_handle *hp, void *stream, int *line) {
    if (!hp || !line) return fail(PLV_ERR_INVALID, "plv_check_status: NULL argument");
    *line = 0;
#if PLV_CHECKED
    PLV_GUARD(&hp->h);
    plv_status st = check_cuda(cudaStreamSynchronize((cudaStream_t)stream),
                               "plv_check_status: sync");
    if (st != PLV_OK) return st;
    for (CheckReader r : check_units()) {
        const int v = r();
        if (v && !*line) *line = v;
    }
#else
    (void)stream;
#endif
    return PLV_OK;
}

int plv_build_checked(void) { return PLV_CHECKED ? 1 : 0; }

plv_status plv_memory_usage(const plv_handle *hp, size_t *current, size_t *peak) {
    if (!hp) return fail(PLV_ERR_INVALID, "plv_memory_usage: NULL handle");
    if (current) *current = hp->h.workspace_used;
    if (peak) *peak = hp->h.workspace_peak;
    return PLV_OK;
}

plv_status plv_debug_fault(int kind, int countdown) {
    (void)g_fault_env_read;
    if (kind == PLV_FAULT_NONE) {
        g_fault_kind.store(PLV_FAULT_NONE);
        g_fault_left.store(0);
        return PLV_OK;
    }
    if (kind != PLV_FAULT_ALLOC && kind != PLV_FAULT_LAUNCH && kind != PLV_FAULT_STALL)
        return fail(PLV_ERR_INVALID, "plv_debug_fault: unknown kind %d", kind);
    if (countdown < 1) return fail(PLV_ERR_INVALID, "plv_debug_fault: countdown %d < 1", countdown);
    g_fault_kind.store(PLV_FAULT_NONE);
    g_fault_left.store(countdown);
    g_fault_kind.store(kind);
    return PLV_OK;
}

int plv_debug_fault_armed(int *countdown) {
    const int k = g_fault_kind.load();
    if (countdown) *countdown = k == PLV_FAULT_NONE ? 0 : g_fault_left.load();
    return k;
}

int64_t plv_phasor_ld(int T) { return T > 0 ? padded_len(T) : 0; }

size_t plv_phasor_bytes(const plv_handle *hp, int batch, int N, int T) {
    if (batch < 0 || N < 0 || T <= 0) return 0;
    const bool split = hp && hp->h.prec != PLV_PREC_FP32;
    const size_t rows = split ? (size_t)row_blocks(N) * kTileRows : (size_t)N;
    return (size_t)batch * rows * (size_t)padded_len(T) * 8u;
}

plv_status plv_prepare(plv_handle *hp, int T) {
    PLV_RANGE("plv_prepare");
    if (!hp) return fail(PLV_ERR_INVALID, "plv_prepare: handle is NULL");
    if (T <= 0) return fail(PLV_ERR_INVALID, "plv_prepare: T = %d", T);
    const int L = log2_exact(T);
    if (L >= kMinLog2T && L <= kMaxLog2Direct) return PLV_OK;  // tables made by plv_create
    PLV_GUARD(&hp->h);
    std::lock_guard<std::mutex> lock(hp->h.mu);
    const ConvPlan *plan = nullptr;
    return get_conv_plan(hp->h, T, &plan);
}

plv_status plv_analytic(plv_handle *hp, void *stream, const void *x,
                        plv_dtype dtype, int batch, int N, int T, int64_t ldx,
                        void *P) {
    PLV_RANGE("plv_analytic");
    if (!hp) return fail(PLV_ERR_INVALID, "plv_analytic: handle is NULL");
    if (batch < 0 || N < 0 || T <= 0)
        return fail(PLV_ERR_INVALID, "plv_analytic: bad sizes batch=%d N=%d T=%d", batch, N, T);
    if (dtype != PLV_F32 && dtype != PLV_F64)
        return fail(PLV_ERR_INVALID, "plv_analytic: unknown dtype %d", (int)dtype);
    if (ldx < T) return fail(PLV_ERR_INVALID, "plv_analytic: ldx %lld < T %d", (long long)ldx, T);
    if (batch == 0 || N == 0) return PLV_OK;
    if (!x || !P) return fail(PLV_ERR_INVALID, "plv_analytic: NULL data pointer");
    const int L = log2_exact(T);
    const bool direct = L >= kMinLog2T && L <= kMaxLog2Direct;
    if (!direct && (T < 2 || 2 * T - 1 > kMaxConvM))
        return fail(PLV_ERR_UNSUPPORTED, "plv_analytic: T = %d (supported: 2 <= T <= %d)", T,
                    kMaxConvM / 2);
    const size_t esz = dtype == PLV_F32 ? 4 : 8;
    if (((uintptr_t)x % esz) != 0)
        return fail(PLV_ERR_INVALID, "plv_analytic: x is not %zu-byte aligned", esz);
    if (((uintptr_t)P % 16) != 0)
        return fail(PLV_ERR_INVALID, "plv_analytic: P is not 16-byte aligned");
    PLV_GUARD(&hp->h);
    if (hp->h.prec != PLV_PREC_FP32) {
        plv_status st = PLV_CHECK_LAUNCH(launch_zero_pad_rows((cudaStream_t)stream, P, batch, N, T),
                                   "plv_analytic: pad rows");
        if (st != PLV_OK) return st;
    }
    if (direct)
        return PLV_CHECK_LAUNCH(launch_analytic_pow2(&hp->h, (cudaStream_t)stream, x, dtype,
                                               (int64_t)batch * N, N, L, ldx, P),
                          "plv_analytic launch");
    const ConvPlan *plan = nullptr;
    {
        std::lock_guard<std::mutex> lock(hp->h.mu);
        if (!hp->h.conv.count(T)) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) == cudaSuccess &&
                cs != cudaStreamCaptureStatusNone)
                return fail(PLV_ERR_INVALID,
                            "plv_analytic: tables for T = %d must be made before capture "
                            "(call plv_prepare)", T);
        }
        plv_status st = get_conv_plan(hp->h, T, &plan);
        if (st != PLV_OK) return st;
    }
    return PLV_CHECK_LAUNCH(launch_analytic_conv(&hp->h, (cudaStream_t)stream, x, dtype,
                                           (int64_t)batch * N, N, T, ldx, P, *plan),
                      "plv_analytic launch");
}

plv_status plv_analytic_bands(plv_handle *hp, void *stream, const void *x, plv_dtype dtype,
                              int batch, int N, int T, int64_t ldx, const float *masks,
                              int nbands, void *P) {
    PLV_RANGE("plv_analytic_bands");
    if (!hp) return fail(PLV_ERR_INVALID, "plv_analytic_bands: handle is NULL");
    if (batch < 0 || N < 0 || T <= 0 || nbands < 0)
        return fail(PLV_ERR_INVALID, "plv_analytic_bands: bad sizes batch=%d N=%d T=%d bands=%d",
                    batch, N, T, nbands);
    if (dtype != PLV_F32 && dtype != PLV_F64)
        return fail(PLV_ERR_INVALID, "plv_analytic_bands: unknown dtype %d", (int)dtype);
    if (ldx < T) return fail(PLV_ERR_INVALID, "plv_analytic_bands: ldx < T");
    const int L = log2_exact(T);
    const bool direct = L >= kMinLog2Bands && L <= kMaxLog2Direct;
    if (!direct && (T < 2 || 2 * T - 1 > kMaxConvM))
        return fail(PLV_ERR_UNSUPPORTED, "plv_analytic_bands: T = %d (2 .. %d)", T,
                    kMaxConvM / 2);
    if (batch == 0 || N == 0 || nbands == 0) return PLV_OK;
    if (!x || !masks || !P) return fail(PLV_ERR_INVALID, "plv_analytic_bands: NULL pointer");
    const size_t esz = dtype == PLV_F32 ? 4 : 8;
    if (((uintptr_t)x % esz) != 0 || ((uintptr_t)masks % 4) != 0 || ((uintptr_t)P % 16) != 0)
        return fail(PLV_ERR_INVALID, "plv_analytic_bands: misaligned pointer");
    PLV_GUARD(&hp->h);
    const size_t band_bytes = plv_phasor_bytes(hp, batch, N, T);
    cudaStream_t s = (cudaStream_t)stream;
    if (!direct) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
            return fail(PLV_ERR_INVALID,
                        "plv_analytic_bands: T = %d is not a power of two from %d to %d, which "
                        "reads the masks back: not inside a capture",
                        T, 1 << kMinLog2Bands, 1 << kMaxLog2Direct);
    }
    if (hp->h.prec != PLV_PREC_FP32)
        for (int b = 0; b < nbands; ++b) {
            plv_status st = PLV_CHECK_LAUNCH(
                launch_zero_pad_rows(s, (uint8_t *)P + (size_t)b * band_bytes, batch, N, T),
                "plv_analytic_bands: pad rows");
            if (st != PLV_OK) return st;
        }
    if (direct)
        return PLV_CHECK_LAUNCH(launch_analytic_bands(&hp->h, s, x, dtype, (int64_t)batch * N, N, L,
                                                ldx, masks, nbands, P, (int64_t)band_bytes),
                          "plv_analytic_bands launch");
    // any other length: the band kernels' spectra are built on the host from
    // the mask values (read back, so the stream is synchronised) and cached;
    // the forward spectrum of each row is kept in the handle's scratch
    Handle &h = hp->h;
    const ConvPlan *plan = nullptr;
    const float2 *K = nullptr;
    std::lock_guard<std::mutex> lock(h.mu);  // the scratch stays as sized through the launch
    plv_status st = get_band_plan(h, s, T, masks, nbands, &plan, &K);
    if (st != PLV_OK) return st;
    st = ensure_workspace(h, s, sizeof(float2) * (size_t)conv_grid(h.num_sms, plan->M) *
                                    (size_t)plan->M);
    if (st != PLV_OK) return st;
    return PLV_CHECK_LAUNCH(launch_analytic_bands_conv(&h, s, x, dtype, (int64_t)batch * N, N, T, ldx,
                                                 *plan, K, nbands, P, (int64_t)band_bytes,
                                                 (float2 *)h.ws),
                      "plv_analytic_bands launch");
}

plv_status plv_normalize(plv_handle *hp, void *stream, const void *z,
                         plv_dtype dtype, int batch, int N, int T, int64_t ldz,
                         void *P) {
    PLV_RANGE("plv_normalize");
    if (!hp) return fail(PLV_ERR_INVALID, "plv_normalize: handle is NULL");
    if (batch < 0 || N < 0 || T <= 0)
        return fail(PLV_ERR_INVALID, "plv_normalize: bad sizes batch=%d N=%d T=%d", batch, N, T);
    if (dtype != PLV_F32 && dtype != PLV_F64)
        return fail(PLV_ERR_INVALID, "plv_normalize: unknown dtype %d", (int)dtype);
    if (ldz < T) return fail(PLV_ERR_INVALID, "plv_normalize: ldz < T");
    if (batch == 0 || N == 0) return PLV_OK;
    if (!z || !P) return fail(PLV_ERR_INVALID, "plv_normalize: NULL data pointer");
    if (((uintptr_t)z % (dtype == PLV_F32 ? 8 : 16)) != 0 || ((uintptr_t)P % 16) != 0)
        return fail(PLV_ERR_INVALID, "plv_normalize: misaligned pointer");
    PLV_GUARD(&hp->h);
    if (hp->h.prec != PLV_PREC_FP32) {
        plv_status st = PLV_CHECK_LAUNCH(launch_zero_pad_rows((cudaStream_t)stream, P, batch, N, T),
                                   "plv_normalize: pad rows");
        if (st != PLV_OK) return st;
    }
    return PLV_CHECK_LAUNCH(launch_normalize(&hp->h, (cudaStream_t)stream, z, dtype,
                                       (int64_t)batch * N, N, T, ldz, P),
                      "plv_normalize launch");
}

plv_status plv_gram(plv_handle *hp, void *stream, const void *P, int batch,
                    int N, int T, unsigned out_mask, float *plv, float *iplv,
                    float *ciplv, void *C, double *diag_dev) {
    PLV_RANGE("plv_gram");
    if (!hp) return fail(PLV_ERR_INVALID, "plv_gram: handle is NULL");
    if (batch < 0 || N < 0 || T <= 0)
        return fail(PLV_ERR_INVALID, "plv_gram: bad sizes batch=%d N=%d T=%d", batch, N, T);
    if (out_mask & ~15u) return fail(PLV_ERR_INVALID, "plv_gram: unknown output bits");
    if (batch == 0 || N == 0) return PLV_OK;
    if (!P) return fail(PLV_ERR_INVALID, "plv_gram: P is NULL");
    if (((uintptr_t)P % 16) != 0) return fail(PLV_ERR_INVALID, "plv_gram: P misaligned");
    GramOut o;
    o.plv = (out_mask & PLV_OUT_PLV) ? plv : nullptr;
    o.iplv = (out_mask & PLV_OUT_IPLV) ? iplv : nullptr;
    o.ciplv = (out_mask & PLV_OUT_CIPLV) ? ciplv : nullptr;
    o.C = (out_mask & PLV_OUT_C) ? (float2 *)C : nullptr;
    o.diag = diag_dev;
    if (o.C && ((uintptr_t)o.C % 8) != 0)
        return fail(PLV_ERR_INVALID, "plv_gram: C is not 8-byte aligned");
    if ((o.plv && ((uintptr_t)o.plv % 4)) || (o.iplv && ((uintptr_t)o.iplv % 4)) ||
        (o.ciplv && ((uintptr_t)o.ciplv % 4)))
        return fail(PLV_ERR_INVALID, "plv_gram: float output not 4-byte aligned");
    o.vec_ok = (N % 4 == 0) && !((uintptr_t)o.plv % 16) && !((uintptr_t)o.iplv % 16) &&
               !((uintptr_t)o.ciplv % 16) && !((uintptr_t)o.C % 16);
    if ((int64_t)N * N > ((int64_t)1 << 40))
        return fail(PLV_ERR_UNSUPPORTED, "plv_gram: N = %d too large", N);
    PLV_GUARD(&hp->h);
    cudaStream_t s = (cudaStream_t)stream;
    if (o.diag) {
        plv_status st = check_cuda(cudaMemsetAsync(o.diag, 0, sizeof(double) * batch, s),
                                   "plv_gram: clear diag");
        if (st != PLV_OK) return st;
    }
    if (hp->h.prec == PLV_PREC_FP32)
        return PLV_CHECK_LAUNCH(launch_gram_fp32(&hp->h, s, (const float *)P, batch, N, T, o),
                          "plv_gram launch");
    return PLV_CHECK_LAUNCH(launch_gram_tc(&hp->h, s, P, batch, N, T, o), "plv_gram launch");
}

plv_status plv_gram_windows(plv_handle *hp, void *stream, const void *P, int batch, int N,
                            int T, int t0, int W, int hop, int nw, unsigned out_mask,
                            float *plv, float *iplv, float *ciplv, void *C, double *diag_dev) {
    PLV_RANGE("plv_gram_windows");
    if (!hp) return fail(PLV_ERR_INVALID, "plv_gram_windows: handle is NULL");
    if (batch < 0 || N < 0 || T <= 0 || nw < 0 || t0 < 0 || W < kTileK || hop < 0 ||
        t0 % kTileK || W % kTileK || hop % kTileK ||
        (nw > 0 && (int64_t)t0 + (int64_t)(nw - 1) * hop + W > T))
        return fail(PLV_ERR_INVALID,
                    "plv_gram_windows: bad windows batch=%d N=%d T=%d t0=%d W=%d hop=%d nw=%d "
                    "(t0, W, hop multiples of %d; windows inside T)",
                    batch, N, T, t0, W, hop, nw, kTileK);
    if (out_mask & ~15u) return fail(PLV_ERR_INVALID, "plv_gram_windows: unknown output bits");
    if (batch == 0 || N == 0 || nw == 0) return PLV_OK;
    if (!P || ((uintptr_t)P % 16) != 0)
        return fail(PLV_ERR_INVALID, "plv_gram_windows: P NULL or misaligned");
    GramOut o;
    o.plv = (out_mask & PLV_OUT_PLV) ? plv : nullptr;
    o.iplv = (out_mask & PLV_OUT_IPLV) ? iplv : nullptr;
    o.ciplv = (out_mask & PLV_OUT_CIPLV) ? ciplv : nullptr;
    o.C = (out_mask & PLV_OUT_C) ? (float2 *)C : nullptr;
    o.diag = diag_dev;
    if ((o.C && ((uintptr_t)o.C % 8)) || (o.plv && ((uintptr_t)o.plv % 4)) ||
        (o.iplv && ((uintptr_t)o.iplv % 4)) || (o.ciplv && ((uintptr_t)o.ciplv % 4)))
        return fail(PLV_ERR_INVALID, "plv_gram_windows: output misaligned");
    o.vec_ok = (N % 4 == 0) && !((uintptr_t)o.plv % 16) && !((uintptr_t)o.iplv % 16) &&
               !((uintptr_t)o.ciplv % 16) && !((uintptr_t)o.C % 16);
    PLV_GUARD(&hp->h);
    cudaStream_t s = (cudaStream_t)stream;
    if (o.diag) {
        plv_status st = check_cuda(cudaMemsetAsync(o.diag, 0, sizeof(double) * batch * nw, s),
                                   "plv_gram_windows: clear diag");
        if (st != PLV_OK) return st;
    }
    if (hp->h.prec == PLV_PREC_FP32)
        return PLV_CHECK_LAUNCH(launch_gram_fp32_windows(&hp->h, s, (const float *)P, batch, N, T, t0,
                                                   W, hop, nw, o),
                          "plv_gram_windows launch");
    return PLV_CHECK_LAUNCH(launch_gram_tc_windows(&hp->h, s, P, batch, N, T, t0, W, hop, nw, o),
                      "plv_gram_windows launch");
}

}  // extern "C"

namespace {

// The analytic-signal part of a plan: descriptors, (problem, pair) items by
// class and decreasing M, padding rows zeroed.  Called with the handle's
// device current.
plv_status plan_k1(Handle &h, const plv_problem *probs, int nprob, plv_group *g) {
    std::vector<K1Desc> descs;
    bool first = true;
    for (int p = 0; p < nprob; ++p) {
        const plv_problem &q = probs[p];
        if (!q.x || q.batch == 0 || q.N == 0) continue;
        if (q.dtype != PLV_F32 && q.dtype != PLV_F64)
            return fail(PLV_ERR_INVALID, "plv_group_create: problem %d unknown dtype", p);
        if (first) g->k1_dtype = q.dtype;
        first = false;
        if (q.dtype != g->k1_dtype)
            return fail(PLV_ERR_UNSUPPORTED,
                        "plv_group_create: problem %d: every input of a plan has one dtype", p);
        if (q.ldx < q.T)
            return fail(PLV_ERR_INVALID, "plv_group_create: problem %d ldx < T", p);
        if (q.T < 2 || 2 * q.T - 1 > kMaxConvM)
            return fail(PLV_ERR_UNSUPPORTED, "plv_group_create: problem %d T = %d (2..%d)", p,
                        q.T, kMaxConvM / 2);
        if (((uintptr_t)q.x % (q.dtype == PLV_F32 ? 4 : 8)) != 0)
            return fail(PLV_ERR_INVALID, "plv_group_create: problem %d x misaligned", p);
        const int64_t pairs = ((int64_t)q.batch * q.N + 1) / 2;
        if (pairs > 0x7fffffffLL)
            return fail(PLV_ERR_UNSUPPORTED, "plv_group_create: problem %d too many rows", p);
        const ConvPlan *plan = nullptr;
        {
            std::lock_guard<std::mutex> lock(h.mu);
            plv_status st = get_conv_plan(h, q.T, &plan);
            if (st != PLV_OK) return st;
        }
        K1Desc d;
        d.x = q.x;
        d.P = q.P;
        d.ldx = q.ldx;
        d.ld = padded_len(q.T);
        d.rows = (int64_t)q.batch * q.N;
        d.N = q.N;
        d.T = q.T;
        d.plan = *plan;
        descs.push_back(d);
    }
    if (descs.empty()) return PLV_OK;
    // items: by class, then decreasing M, then problem order
    std::vector<int2> items;
    K1Group kg{};
    k1_layout(descs, g->cfg.k1_class, items, kg);
    plv_status st = check_alloc(dev_malloc(&g->k1_descs, sizeof(K1Desc) * descs.size()),
                               "plv_group_create: analytic descriptors");
    if (st == PLV_OK)
        st = check_alloc(dev_malloc(&g->k1_items, sizeof(int2) * items.size()),
                        "plv_group_create: analytic items");
    if (st == PLV_OK)
        st = check_cuda(cudaMemcpy(g->k1_descs, descs.data(), sizeof(K1Desc) * descs.size(),
                                   cudaMemcpyHostToDevice),
                        "plv_group_create: upload analytic descriptors");
    if (st == PLV_OK)
        st = check_cuda(cudaMemcpy(g->k1_items, items.data(), sizeof(int2) * items.size(),
                                   cudaMemcpyHostToDevice),
                        "plv_group_create: upload analytic items");
    if (st != PLV_OK) return st;
    // the split layout's padding rows: zero once, nothing writes them later
    if (h.prec != PLV_PREC_FP32) {
        for (int p = 0; p < nprob && st == PLV_OK; ++p) {
            const plv_problem &q = probs[p];
            if (!q.x || q.batch == 0 || q.N == 0) continue;
            st = PLV_CHECK_LAUNCH(launch_zero_pad_rows(0, q.P, q.batch, q.N, q.T),
                            "plv_group_create: padding rows");
        }
        if (st == PLV_OK)
            st = check_cuda(cudaDeviceSynchronize(), "plv_group_create: padding rows");
        if (st != PLV_OK) return st;
    }
    kg.descs = g->k1_descs;
    kg.items = g->k1_items;
    g->k1 = kg;
    g->k1_host = std::move(descs);
    g->has_k1 = true;
    return PLV_OK;
}

}  // namespace

extern "C" {

plv_status plv_group_create(plv_handle *hp, const plv_problem *probs, int nprob,
                            unsigned out_mask, plv_group **out) {
    PLV_RANGE("plv_group_create");
    if (!hp || !out) return fail(PLV_ERR_INVALID, "plv_group_create: NULL argument");
    *out = nullptr;
    if (nprob < 0 || (nprob > 0 && !probs))
        return fail(PLV_ERR_INVALID, "plv_group_create: bad problem list");
    if (out_mask & ~15u) return fail(PLV_ERR_INVALID, "plv_group_create: unknown output bits");
    Handle &h = hp->h;
    plv_group *g = new (std::nothrow) plv_group();
    if (!g) return fail(PLV_ERR_ALLOC, "plv_group_create: out of host memory");
    g->device = h.device;
    g->prec = h.prec;
    g->mask = out_mask;
    std::vector<TcProblem> dp;
    std::vector<int4> items;
    for (int p = 0; p < nprob; ++p) {
        plv_problem q = probs[p];
        if (q.batch < 0 || q.N < 0 || q.T <= 0) {
            delete g;
            return fail(PLV_ERR_INVALID, "plv_group_create: problem %d has bad sizes", p);
        }
        if (q.batch == 0 || q.N == 0) continue;
        if (!q.P || ((uintptr_t)q.P % 16) != 0) {
            delete g;
            return fail(PLV_ERR_INVALID, "plv_group_create: problem %d phasors NULL or misaligned", p);
        }
        if (!(out_mask & PLV_OUT_PLV)) q.plv = nullptr;
        if (!(out_mask & PLV_OUT_IPLV)) q.iplv = nullptr;
        if (!(out_mask & PLV_OUT_CIPLV)) q.ciplv = nullptr;
        if (!(out_mask & PLV_OUT_C)) q.C = nullptr;
        if ((q.C && ((uintptr_t)q.C % 8)) || (q.plv && ((uintptr_t)q.plv % 4)) ||
            (q.iplv && ((uintptr_t)q.iplv % 4)) || (q.ciplv && ((uintptr_t)q.ciplv % 4))) {
            delete g;
            return fail(PLV_ERR_INVALID, "plv_group_create: problem %d output misaligned", p);
        }
        if (q.diag) g->any_diag = true;
        g->host.push_back(q);
        GramOut o;
        o.plv = q.plv;
        o.iplv = q.iplv;
        o.ciplv = q.ciplv;
        o.C = (float2 *)q.C;
        o.diag = q.diag;
        o.vec_ok = (q.N % 4 == 0) && !((uintptr_t)o.plv % 16) && !((uintptr_t)o.iplv % 16) &&
                   !((uintptr_t)o.ciplv % 16) && !((uintptr_t)o.C % 16);
        const TcProblem tp = make_tc_problem(q.P, q.batch, q.N, q.T, o);
        if (tp.nrb > 0xffff) {  // tile coordinates are 16-bit in the launch list
            delete g;
            return fail(PLV_ERR_UNSUPPORTED, "plv_group_create: problem %d N = %d too large", p,
                        q.N);
        }
        const int pid = (int)dp.size();
        dp.push_back(tp);
        for (int e = 0; e < q.batch; ++e)
            for (int J = 0; J < tp.nrb; ++J)
                for (int I = 0; I <= J; ++I) items.push_back(make_int4(pid, e, I, J));
    }
    if (items.size() > 0x7fffffffu) {
        delete g;
        return fail(PLV_ERR_UNSUPPORTED, "plv_group_create: too many tiles");
    }
    {
        DeviceGuard guard(h.device);
        plv_status st = plan_k1(h, probs, nprob, g);
        if (st != PLV_OK) {
            plv_group_destroy(g);
            return st;
        }
    }
    // longest first: a tile's cost is proportional to its K blocks
    std::stable_sort(items.begin(), items.end(), [&](const int4 &a, const int4 &b) {
        return dp[a.x].nkb > dp[b.x].nkb;
    });
    g->dp_host = dp;
    g->items_host = items;
    g->nprob = (int)dp.size();
    g->ntiles = (int)items.size();
    g->nitems = g->ntiles;
    if (h.prec != PLV_PREC_FP32 && g->nprob > 0) {
        DeviceGuard guard(h.device);
        plv_status st = check_alloc(dev_malloc(&g->probs, sizeof(TcProblem) * dp.size()),
                                   "plv_group_create: descriptors");
        if (st == PLV_OK)
            st = check_cuda(cudaMemcpy(g->probs, dp.data(), sizeof(TcProblem) * dp.size(),
                                       cudaMemcpyHostToDevice),
                            "plv_group_create: upload descriptors");
        if (st == PLV_OK && g->ntiles > 0) {
            // the default launch list: longest first, no tile split
            const GramList list = gram_list(dp, items, gram_chunk_kb(h.prec), h.num_sms, g->cfg);
            st = upload_list(list, nullptr, &g->items, &g->split);
            if (st == PLV_OK) g->nitems = (int)list.items.size();
        }
        if (st != PLV_OK) {
            plv_group_destroy(g);
            return st;
        }
    }
    *out = g;
    return PLV_OK;
}

plv_status plv_gram_grouped(plv_handle *hp, void *stream, const plv_group *g) {
    PLV_RANGE("plv_gram_grouped");
    if (!hp || !g) return fail(PLV_ERR_INVALID, "plv_gram_grouped: NULL argument");
    if (g->device != hp->h.device || g->prec != hp->h.prec)
        return fail(PLV_ERR_INVALID, "plv_gram_grouped: plan made for another device or precision");
    PLV_GUARD(&hp->h);
    cudaStream_t s = (cudaStream_t)stream;
    if (hp->h.prec == PLV_PREC_FP32) {
        for (const plv_problem &q : g->host) {
            plv_status st = plv_gram(hp, stream, q.P, q.batch, q.N, q.T, g->mask, q.plv, q.iplv,
                                     q.ciplv, q.C, q.diag);
            if (st != PLV_OK) return st;
        }
        return PLV_OK;
    }
    if (g->nitems == 0) return PLV_OK;
    if (g->any_diag) {
        plv_status st = PLV_CHECK_LAUNCH(launch_zero_group_diag(s, g->probs, g->nprob),
                                   "plv_gram_grouped: clear diag");
        if (st != PLV_OK) return st;
    }
    if (g->split.ntiles > 0) {
        // split tiles count their chunks from zero in every launch
        plv_status st = check_cuda(cudaMemsetAsync(g->split.counters, 0,
                                                   sizeof(int) * 16 * (size_t)g->split.ntiles, s),
                                   "plv_gram_grouped: split counters");
        if (st != PLV_OK) return st;
    }
    return PLV_CHECK_LAUNCH(
        launch_gram_tc_group(&hp->h, s, g->probs, g->items, g->nitems, g->split),
        "plv_gram_grouped launch");
}

plv_status plv_analytic_grouped(plv_handle *hp, void *stream, const plv_group *g) {
    PLV_RANGE("plv_analytic_grouped");
    if (!hp || !g) return fail(PLV_ERR_INVALID, "plv_analytic_grouped: NULL argument");
    if (g->device != hp->h.device || g->prec != hp->h.prec)
        return fail(PLV_ERR_INVALID,
                    "plv_analytic_grouped: plan made for another device or precision");
    if (!g->has_k1) return fail(PLV_ERR_INVALID, "plv_analytic_grouped: the plan has no input");
    PLV_GUARD(&hp->h);
    return PLV_CHECK_LAUNCH(launch_analytic_group(&hp->h, (cudaStream_t)stream, g->k1_dtype, g->k1),
                      "plv_analytic_grouped launch");
}

plv_status plv_group_destroy(plv_group *g) {
    PLV_RANGE("plv_group_destroy");
    if (!g) return PLV_OK;
    {
        DeviceGuard guard(g->device);
        if (g->probs || g->items || g->k1_descs || g->k1_items || !g->retired.empty())
            cudaDeviceSynchronize();
        if (g->probs) cudaFree(g->probs);
        free_list(g->items, g->split);
        if (g->k1_descs) cudaFree(g->k1_descs);
        if (g->k1_items) cudaFree(g->k1_items);
        for (void *p : g->retired)
            if (p) cudaFree(p);
    }
    delete g;
    return PLV_OK;
}

plv_status plv_trial_operands(plv_handle *hp, void *stream, const float *V, int E, int N,
                              int64_t ldv, int l0, int L, int mode, void *P) {
    PLV_RANGE("plv_trial_operands");
    if (!hp) return fail(PLV_ERR_INVALID, "plv_trial_operands: handle is NULL");
    if (E < 1 || N < 0 || L < 0 || l0 < 0 || ldv < 0 || (int64_t)l0 + L > ldv)
        return fail(PLV_ERR_INVALID, "plv_trial_operands: bad sizes E=%d N=%d ldv=%lld l0=%d L=%d",
                    E, N, (long long)ldv, l0, L);
    if (mode != PLV_TRIAL_ASIS && mode != PLV_TRIAL_RMS)
        return fail(PLV_ERR_INVALID, "plv_trial_operands: unknown mode %d", mode);
    if (N > 65408) return fail(PLV_ERR_UNSUPPORTED, "plv_trial_operands: N = %d > 65408", N);
    if (N == 0 || L == 0) return PLV_OK;
    if (!V || !P) return fail(PLV_ERR_INVALID, "plv_trial_operands: NULL pointer");
    if (((uintptr_t)V % 4) != 0 || ((uintptr_t)P % 16) != 0)
        return fail(PLV_ERR_INVALID, "plv_trial_operands: misaligned pointer");
    PLV_GUARD(&hp->h);
    return PLV_CHECK_LAUNCH(launch_trial_operands(&hp->h, (cudaStream_t)stream, V, E, N, ldv, l0, L,
                                            mode == PLV_TRIAL_RMS, P),
                      "plv_trial_operands launch");
}

plv_status plv_dft_bins(plv_handle *hp, void *stream, const void *x, plv_dtype dtype, int rows,
                        int T, int64_t ldx, int f0, int F, float *X, int64_t ldX) {
    PLV_RANGE("plv_dft_bins");
    if (!hp) return fail(PLV_ERR_INVALID, "plv_dft_bins: handle is NULL");
    if (dtype != PLV_F32 && dtype != PLV_F64)
        return fail(PLV_ERR_INVALID, "plv_dft_bins: unknown dtype %d", (int)dtype);
    if (rows < 0 || T < 1 || T > 32768 || ldx < T || f0 < 0 || F < 1 || f0 + F > T || ldX < F)
        return fail(PLV_ERR_INVALID,
                    "plv_dft_bins: bad sizes rows=%d T=%d ldx=%lld f0=%d F=%d ldX=%lld", rows, T,
                    (long long)ldx, f0, F, (long long)ldX);
    if (rows == 0) return PLV_OK;
    if (!x || !X) return fail(PLV_ERR_INVALID, "plv_dft_bins: NULL pointer");
    if (((uintptr_t)x % (dtype == PLV_F32 ? 4 : 8)) != 0 || ((uintptr_t)X % 4) != 0)
        return fail(PLV_ERR_INVALID, "plv_dft_bins: misaligned pointer");
    PLV_GUARD(&hp->h);
    return PLV_CHECK_LAUNCH(launch_dft_bins((cudaStream_t)stream, x, dtype, rows, T, ldx, f0, F, X, ldX),
                      "plv_dft_bins launch");
}

plv_status plv_metrics(plv_handle *hp, void *stream, const void *C, int batch,
                       int N, float *plv, float *iplv, float *ciplv) {
    PLV_RANGE("plv_metrics");
    if (!hp) return fail(PLV_ERR_INVALID, "plv_metrics: handle is NULL");
    if (batch < 0 || N < 0) return fail(PLV_ERR_INVALID, "plv_metrics: bad sizes");
    if (batch == 0 || N == 0) return PLV_OK;
    if (!C) return fail(PLV_ERR_INVALID, "plv_metrics: C is NULL");
    if (((uintptr_t)C % 8) != 0) return fail(PLV_ERR_INVALID, "plv_metrics: C misaligned");
    PLV_GUARD(&hp->h);
    return PLV_CHECK_LAUNCH(launch_metrics((cudaStream_t)stream, (const float2 *)C, batch, N,
                                     plv, iplv, ciplv),
                      "plv_metrics launch");
}

plv_status plv_backward(plv_handle *hp, void *stream, const void *x, plv_dtype dtype,
                        int batch, int N, int T, int64_t ldx, const void *C,
                        const float *g_plv, const float *g_iplv, const float *g_ciplv,
                        float *grad_x) {
    PLV_RANGE("plv_backward");
    if (!hp) return fail(PLV_ERR_INVALID, "plv_backward: handle is NULL");
    if (batch < 0 || N < 0 || T <= 0)
        return fail(PLV_ERR_INVALID, "plv_backward: bad sizes batch=%d N=%d T=%d", batch, N, T);
    if (dtype != PLV_F32 && dtype != PLV_F64)
        return fail(PLV_ERR_INVALID, "plv_backward: unknown dtype %d", (int)dtype);
    if (ldx < T) return fail(PLV_ERR_INVALID, "plv_backward: ldx < T");
    if (batch == 0 || N == 0) return PLV_OK;
    if (!grad_x) return fail(PLV_ERR_INVALID, "plv_backward: grad_x is NULL");
    const int L = log2_exact(T);
    const bool direct = L >= kMinLog2T && L <= kMaxLog2Direct;
    if (!direct && (T < 2 || 2 * T - 1 > kMaxConvM))
        return fail(PLV_ERR_UNSUPPORTED, "plv_backward: T = %d (supported: 2 <= T <= %d)", T,
                    kMaxConvM / 2);
    PLV_GUARD(&hp->h);
    Handle &h = hp->h;
    cudaStream_t s = (cudaStream_t)stream;
    if (!g_plv && !g_iplv && !g_ciplv)
        return check_cuda(cudaMemsetAsync(grad_x, 0, sizeof(float) * (size_t)batch * N * T, s),
                          "plv_backward: zero grad");
    if (!x || !C) return fail(PLV_ERR_INVALID, "plv_backward: NULL x or C");
    if (((uintptr_t)C % 8) != 0 || ((uintptr_t)x % (dtype == PLV_F32 ? 4 : 8)) != 0 ||
        ((uintptr_t)grad_x % 4) != 0)
        return fail(PLV_ERR_INVALID, "plv_backward: misaligned pointer");
    const int64_t ld = padded_len(T);
    const size_t rows = (size_t)batch * N;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // split-precision handles take the contraction to the tensor cores; their
    // S (split rows) and conj(P)^T operands replace the FP32 S
    const bool tc = h.prec != PLV_PREC_FP32;
    const size_t bP = up(rows * 2 * ld * 4), bR = up(rows * ld * 4), bG = up(rows * 2 * ld * 4),
                 bS = tc ? up(backward_tc_bytes(batch, N, T, nullptr))
                         : up((size_t)batch * 2 * N * N * 4);
    std::lock_guard<std::mutex> lock(h.mu);
    plv_status st = ensure_workspace(h, s, bP + bR + bG + bS);
    if (st != PLV_OK) return st;
    const ConvPlan *plan = nullptr;
    if (!direct) {
        if (!h.conv.count(T)) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
                return fail(PLV_ERR_INVALID,
                            "plv_backward: tables for T = %d must be made before capture "
                            "(call plv_prepare)", T);
        }
        st = get_conv_plan(h, T, &plan);
        if (st != PLV_OK) return st;
    }
    char *w = (char *)h.ws;
    float *P = (float *)w, *rinv = (float *)(w + bP), *Gm = (float *)(w + bP + bR),
          *S = (float *)(w + bP + bR + bG);
    // split-precision handles: the recompute also writes P's BF16 splits, the
    // contraction's B operand, whose padding rows N .. 128 ceil(N/128) - 1
    // must be zero (the scratch is shared with other calls)
    void *Ps = nullptr;
    if (tc) {
        size_t a_bytes = 0;
        backward_tc_bytes(batch, N, T, &a_bytes);
        Ps = (char *)S + a_bytes;
        if (N % 128 != 0) {
            st = PLV_CHECK_LAUNCH(launch_zero_pad_rows(s, Ps, batch, N, T),
                                  "plv_backward: padding rows");
            if (st != PLV_OK) return st;
        }
    }
    st = PLV_CHECK_LAUNCH(launch_bwd_prep(&h, s, x, dtype, (int64_t)rows, L, ldx, P, rinv, T, plan,
                                          Ps, N),
                    "plv_backward: recompute");
    if (st != PLV_OK) return st;
    return PLV_CHECK_LAUNCH(launch_backward(&h, s, batch, N, T, L, (const float2 *)C, g_plv, g_iplv,
                                      g_ciplv, P, rinv, tc ? nullptr : S, Gm, grad_x, plan,
                                      tc ? (void *)S : nullptr, Ps),
                      "plv_backward launch");
}

// The any-length plan for T, made outside stream capture (shared by the
// saved-signal entry points).
static plv_status conv_plan_for(Handle &h, cudaStream_t s, int T, const char *who,
                                const ConvPlan **plan) {
    if (!h.conv.count(T)) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            return fail(PLV_ERR_INVALID,
                        "%s: tables for T = %d must be made before capture (call plv_prepare)",
                        who, T);
    }
    return get_conv_plan(h, T, plan);
}

plv_status plv_analytic_save(plv_handle *hp, void *stream, const void *x, plv_dtype dtype,
                             int batch, int N, int T, int64_t ldx, void *P, float *P32,
                             float *rinv) {
    PLV_RANGE("plv_analytic_save");
    if (!hp) return fail(PLV_ERR_INVALID, "plv_analytic_save: handle is NULL");
    if (batch < 0 || N < 0 || T <= 0)
        return fail(PLV_ERR_INVALID, "plv_analytic_save: bad sizes batch=%d N=%d T=%d", batch, N,
                    T);
    if (dtype != PLV_F32 && dtype != PLV_F64)
        return fail(PLV_ERR_INVALID, "plv_analytic_save: unknown dtype %d", (int)dtype);
    if (ldx < T) return fail(PLV_ERR_INVALID, "plv_analytic_save: ldx < T");
    Handle &h = hp->h;
    if (h.prec == PLV_PREC_FP16X3)
        return fail(PLV_ERR_UNSUPPORTED, "plv_analytic_save: FP16X3 handles (use plv_analytic "
                                         "and plv_backward)");
    if (batch == 0 || N == 0) return PLV_OK;
    const bool fp32 = h.prec == PLV_PREC_FP32;
    if (fp32 && !P32) P32 = (float *)P;
    if (!x || !P || !P32 || !rinv)
        return fail(PLV_ERR_INVALID, "plv_analytic_save: NULL data pointer");
    if (fp32 && (void *)P32 != P)
        return fail(PLV_ERR_INVALID, "plv_analytic_save: on an FP32 handle P32 is P (or NULL)");
    const int L = log2_exact(T);
    const bool direct = L >= kMinLog2T && L <= kMaxLog2Direct;
    if (!direct && (T < 2 || 2 * T - 1 > kMaxConvM))
        return fail(PLV_ERR_UNSUPPORTED, "plv_analytic_save: T = %d (supported: 2 <= T <= %d)",
                    T, kMaxConvM / 2);
    if (((uintptr_t)x % (dtype == PLV_F32 ? 4 : 8)) != 0 || ((uintptr_t)P % 16) != 0 ||
        ((uintptr_t)P32 % 16) != 0 || ((uintptr_t)rinv % 16) != 0)
        return fail(PLV_ERR_INVALID, "plv_analytic_save: misaligned pointer");
    PLV_GUARD(&h);
    cudaStream_t s = (cudaStream_t)stream;
    const ConvPlan *plan = nullptr;
    if (!direct) {
        std::lock_guard<std::mutex> lock(h.mu);
        plv_status st = conv_plan_for(h, s, T, "plv_analytic_save", &plan);
        if (st != PLV_OK) return st;
    }
    if (!fp32) {
        plv_status st = PLV_CHECK_LAUNCH(launch_zero_pad_rows(s, P, batch, N, T),
                                         "plv_analytic_save: pad rows");
        if (st != PLV_OK) return st;
    }
    return PLV_CHECK_LAUNCH(launch_bwd_prep(&h, s, x, dtype, (int64_t)batch * N, L, ldx, P32,
                                            rinv, T, plan, fp32 ? nullptr : P, N),
                            "plv_analytic_save launch");
}

plv_status plv_backward_saved(plv_handle *hp, void *stream, int batch, int N, int T,
                              const void *P, const float *P32, const float *rinv, const void *C,
                              const float *g_plv, const float *g_iplv, const float *g_ciplv,
                              float *grad_x) {
    PLV_RANGE("plv_backward_saved");
    if (!hp) return fail(PLV_ERR_INVALID, "plv_backward_saved: handle is NULL");
    if (batch < 0 || N < 0 || T <= 0)
        return fail(PLV_ERR_INVALID, "plv_backward_saved: bad sizes batch=%d N=%d T=%d", batch,
                    N, T);
    Handle &h = hp->h;
    if (h.prec == PLV_PREC_FP16X3)
        return fail(PLV_ERR_UNSUPPORTED, "plv_backward_saved: FP16X3 handles");
    if (batch == 0 || N == 0) return PLV_OK;
    if (!grad_x) return fail(PLV_ERR_INVALID, "plv_backward_saved: grad_x is NULL");
    const int L = log2_exact(T);
    const bool direct = L >= kMinLog2T && L <= kMaxLog2Direct;
    if (!direct && (T < 2 || 2 * T - 1 > kMaxConvM))
        return fail(PLV_ERR_UNSUPPORTED, "plv_backward_saved: T = %d (supported: 2 <= T <= %d)",
                    T, kMaxConvM / 2);
    PLV_GUARD(&h);
    cudaStream_t s = (cudaStream_t)stream;
    if (!g_plv && !g_iplv && !g_ciplv)
        return check_cuda(cudaMemsetAsync(grad_x, 0, sizeof(float) * (size_t)batch * N * T, s),
                          "plv_backward_saved: zero grad");
    const bool tc = h.prec != PLV_PREC_FP32;
    if (!tc && !P32) P32 = (const float *)P;
    if (!P || !P32 || !rinv || !C)
        return fail(PLV_ERR_INVALID, "plv_backward_saved: NULL P, P32, rinv or C");
    if (((uintptr_t)C % 8) != 0 || ((uintptr_t)P % 16) != 0 || ((uintptr_t)P32 % 16) != 0 ||
        ((uintptr_t)rinv % 16) != 0 || ((uintptr_t)grad_x % 4) != 0)
        return fail(PLV_ERR_INVALID, "plv_backward_saved: misaligned pointer");
    const int64_t ld = padded_len(T);
    const size_t rows = (size_t)batch * N;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t a_bytes = 0;
    if (tc) backward_tc_bytes(batch, N, T, &a_bytes);
    const size_t bG = up(rows * 2 * ld * 4),
                 bS = tc ? up(a_bytes) : up((size_t)batch * 2 * N * N * 4);
    std::lock_guard<std::mutex> lock(h.mu);
    plv_status st = ensure_workspace(h, s, bG + bS);
    if (st != PLV_OK) return st;
    const ConvPlan *plan = nullptr;
    if (!direct) {
        st = conv_plan_for(h, s, T, "plv_backward_saved", &plan);
        if (st != PLV_OK) return st;
    }
    char *w = (char *)h.ws;
    float *Gm = (float *)w, *S = (float *)(w + bG);
    return PLV_CHECK_LAUNCH(launch_backward(&h, s, batch, N, T, L, (const float2 *)C, g_plv,
                                            g_iplv, g_ciplv, P32, rinv, tc ? nullptr : S, Gm,
                                            grad_x, plan, tc ? (void *)S : nullptr,
                                            tc ? P : nullptr),
                            "plv_backward_saved launch");
}

plv_status plv_sync_status(plv_handle *hp, void *stream, int *device_status) {
    PLV_RANGE("plv_sync_status");
    if (!hp || !device_status) return fail(PLV_ERR_INVALID, "plv_sync_status: NULL argument");
    PLV_GUARD(&hp->h);
    cudaStream_t s = (cudaStream_t)stream;
    int v = 0;
    plv_status st = check_cuda(cudaMemcpyAsync(&v, hp->h.status, sizeof(int),
                                               cudaMemcpyDeviceToHost, s),
                               "plv_sync_status: read");
    if (st == PLV_OK) st = check_cuda(cudaStreamSynchronize(s), "plv_sync_status: sync");
    if (st == PLV_OK && v != 0)
        st = check_cuda(cudaMemsetAsync(hp->h.status, 0, sizeof(int), s),
                        "plv_sync_status: clear");
    *device_status = v;
    return st;
}

}  // extern "C"
