// common.cuh -- internal declarations shared by the library's translation
// units: the handle, status helpers, the operand layouts and the kernel
// launchers.  Nothing here is part of the public ABI (include/plv.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>

#include "plv.h"

namespace plv {

// Phasor operand rows are padded to a multiple of this many samples (the
// Gram's K tile); the padding holds zeros.
constexpr int kPadT = 32;

inline int64_t padded_len(int T) {
    return ((int64_t)T + kPadT - 1) / kPadT * kPadT;
}

// Smallest and largest power-of-two lengths the shared-memory FFT handles.
constexpr int kMinLog2T = 5;
constexpr int kMaxLog2T = 14;

// Device status codes written by kernels into the handle's status word.
enum : int { kDevOk = 0, kDevTimeout = 5 };

struct Handle {
    int device = 0;
    plv_precision prec = PLV_PREC_FP32;
    size_t workspace_limit = 0;
    size_t workspace_used = 0;
    int num_sms = 0;
    // twiddles exp(-2 pi i m / 2^L), m < 2^L, for L = kMinLog2T..kMaxLog2T,
    // table L starting at element (2^L - 2^kMinLog2T)
    float2 *twiddles = nullptr;
    int *status = nullptr;  // device status word
    void *ws = nullptr;     // scratch for the backward pass (grows on demand)
    size_t ws_bytes = 0;
    std::mutex mu;
};

// Per-thread last error message.
void set_error(const char *fmt, ...);
plv_status fail(plv_status s, const char *fmt, ...);
plv_status check_cuda(cudaError_t e, const char *what);

inline const float2 *twiddle_table(const Handle *h, int log2T) {
    return h->twiddles + ((1 << log2T) - (1 << kMinLog2T));
}

// ---- kernel launchers (one translation unit each) --------------------------

// K1: fused Hilbert FFT + normalisation, power-of-two T.
cudaError_t launch_analytic_pow2(const Handle *h, cudaStream_t s,
                                 const void *x, plv_dtype dt, int64_t rows,
                                 int N, int log2T, int64_t ldx, void *P);
// Backward preparation: FP32 phasors P[rows][2][ld] and rinv[rows][ld].
cudaError_t launch_bwd_prep(const Handle *h, cudaStream_t s, const void *x, plv_dtype dt,
                            int64_t rows, int log2T, int64_t ldx, float *P, float *rinv);
// K5: S = G + G^H, Gamma = S P / T, grad = Re Gamma_z - H{Im Gamma_z}.
cudaError_t launch_backward(const Handle *h, cudaStream_t st, int batch, int N, int T,
                            int log2T, const float2 *C, const float *g1, const float *g2,
                            const float *g3, const float *P, const float *rinv, float *S,
                            float *Gm, float *grad);
// Eq. 4 on a given analytic signal.
cudaError_t launch_normalize(const Handle *h, cudaStream_t s, const void *z,
                             plv_dtype dt, int64_t rows, int N, int T,
                             int64_t ldz, void *P);
// K2: FP32 SIMT Gram + fused read-outs.
struct GramOut {
    float *plv, *iplv, *ciplv;
    float2 *C;
    double *diag;
    bool vec_ok;  // N % 4 == 0 and every output 16-byte aligned
};
cudaError_t launch_gram_fp32(const Handle *h, cudaStream_t s, const float *P,
                             int batch, int N, int T, GramOut out);
// K3: split-precision tensor-core Gram + fused read-outs (BF16X3 / FP16X3).
cudaError_t launch_gram_tc(const Handle *h, cudaStream_t s, const void *P,
                           int batch, int N, int T, GramOut out);
// K6: read-outs from a stored C.
cudaError_t launch_metrics(cudaStream_t s, const float2 *C, int batch, int N,
                           float *plv, float *iplv, float *ciplv);

}  // namespace plv

struct plv_handle {
    plv::Handle h;
};
