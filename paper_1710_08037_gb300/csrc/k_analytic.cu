// k_analytic.cu -- K1 host dispatch: the analytic signal (Eq. 3) fused with
// the unit-phasor normalisation (Eq. 4) by input type and operand precision
// (the engine launchers are compiled per pair in k_fwd.cu), the zeroing of the
// split layout's padding rows, and Eq. 4 alone on a caller's analytic signal.
#include "analytic.cuh"

namespace plv {
namespace {

// Zero the rows N .. NRB*128-1 of every epoch's last row block, all planes
// and samples: one thread per 16-byte chunk.
__global__ void k_zero_pad_rows(uint4 *P, int batch, int N, int64_t NRB, int64_t NKB) {
    const int pad0 = N & 127;  // first padding row inside the last block
    const int npad = 128 - pad0;
    const int64_t chunks_per_row = kTileK * 2 / 16;  // 4 chunks of 16 bytes
    const int64_t per_block = 4 * (int64_t)npad * chunks_per_row;
    const int64_t total = (int64_t)batch * NKB * per_block;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = q % chunks_per_row;
        int64_t rest = q / chunks_per_row;
        const int64_t rr = rest % npad;
        rest /= npad;
        const int64_t plane = rest % 4;
        rest /= 4;
        const int64_t kb = rest % NKB;
        const int64_t e = rest / NKB;
        const int64_t blk = (e * NRB + (NRB - 1)) * NKB + kb;
        const int64_t el = blk * kBlockElems + plane * (kTileRows * kTileK) +
                           (pad0 + rr) * kTileK + c * 8;
        P[el / 8] = make_uint4(0u, 0u, 0u, 0u);
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
    store_phasor<PREC>(P, row_addr<PREC>(r, N, ld), ld, (int)m, p);
}

// Run F<Tin, KIND> for the handle's precision and the input dtype.
template <template <typename, int> class F, typename... A>
cudaError_t by_kind(plv_precision prec, plv_dtype dt, A &&...args) {
    if (prec == PLV_PREC_FP32)
        return dt == PLV_F32 ? F<float, kK1Fp32>::run(args...) : F<double, kK1Fp32>::run(args...);
    if (prec == PLV_PREC_FP16X3)
        return dt == PLV_F32 ? F<float, kK1Fp16>::run(args...) : F<double, kK1Fp16>::run(args...);
    return dt == PLV_F32 ? F<float, kK1Bf16>::run(args...) : F<double, kK1Bf16>::run(args...);
}
template <typename Tin, int KIND>
struct Pow2 {
    static cudaError_t run(const Handle *h, cudaStream_t s, const K1Args &a) {
        return k1_pow2<Tin, KIND>(h, s, a);
    }
};
template <typename Tin, int KIND>
struct Conv {
    static cudaError_t run(const Handle *h, cudaStream_t s, const K1Args &a, const ConvPlan &p) {
        return k1_conv<Tin, KIND>(h, s, a, p);
    }
};
template <typename Tin, int KIND>
struct Bands {
    static cudaError_t run(const Handle *h, cudaStream_t s, const void *x, int64_t ldx, int N,
                           int64_t rows, int log2T, const float *masks, int nbands, void *P,
                           int64_t band_bytes) {
        return launch_bands<Tin, KIND>(h, s, (const Tin *)x, ldx, N, rows, log2T, masks, nbands,
                                       P, band_bytes);
    }
};
template <typename Tin, int KIND>
struct BandsConv {
    static cudaError_t run(const Handle *h, cudaStream_t s, const void *x, int64_t ldx, int N,
                           int64_t rows, int T, const ConvPlan &plan, const float2 *K,
                           int nbands, void *P, int64_t band_bytes, float2 *scratch) {
        return launch_bands_conv<Tin, KIND>(h, s, (const Tin *)x, ldx, N, rows, T, plan, K,
                                            nbands, P, band_bytes, scratch);
    }
};
template <typename Tin, int KIND>
struct Group {
    static cudaError_t run(const Handle *h, cudaStream_t s, const K1Group &g) {
        return k1_conv_group<Tin, KIND>(h, s, g);
    }
};

}  // namespace

cudaError_t launch_zero_pad_rows(cudaStream_t s, void *P, int batch, int N, int T) {
    if ((N & 127) == 0 || batch == 0) return cudaSuccess;
    const int64_t NKB = padded_len(T) / kTileK;
    const int64_t total = (int64_t)batch * NKB * 4 * (128 - (N & 127)) * 4;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_zero_pad_rows<<<(unsigned)blocks, 256, 0, s>>>((uint4 *)P, batch, N, row_blocks(N), NKB);
    return cudaGetLastError();
}

cudaError_t launch_analytic_conv(const Handle *h, cudaStream_t s, const void *x,
                                 plv_dtype dt, int64_t rows, int N, int T, int64_t ldx,
                                 void *P, const ConvPlan &plan) {
    const K1Args a{x, ldx, P, nullptr, N, T, 0, padded_len(T), rows};
    return by_kind<Conv>(h->prec, dt, h, s, a, plan);
}

cudaError_t launch_analytic_pow2(const Handle *h, cudaStream_t s,
                                 const void *x, plv_dtype dt, int64_t rows,
                                 int N, int log2T, int64_t ldx, void *P) {
    const K1Args a{x, ldx, P, nullptr, N, 1 << log2T, log2T, (int64_t)1 << log2T, rows};
    return by_kind<Pow2>(h->prec, dt, h, s, a);
}

cudaError_t launch_analytic_bands(const Handle *h, cudaStream_t s, const void *x, plv_dtype dt,
                                  int64_t rows, int N, int log2T, int64_t ldx, const float *masks,
                                  int nbands, void *P, int64_t band_bytes) {
    return by_kind<Bands>(h->prec, dt, h, s, x, ldx, N, rows, log2T, masks, nbands, P,
                          band_bytes);
}

cudaError_t launch_analytic_bands_conv(const Handle *h, cudaStream_t s, const void *x,
                                       plv_dtype dt, int64_t rows, int N, int T, int64_t ldx,
                                       const ConvPlan &plan, const float2 *K, int nbands,
                                       void *P, int64_t band_bytes, float2 *scratch) {
    return by_kind<BandsConv>(h->prec, dt, h, s, x, ldx, N, rows, T, plan, K, nbands, P,
                              band_bytes, scratch);
}

cudaError_t launch_analytic_group(const Handle *h, cudaStream_t s, plv_dtype dt,
                                  const K1Group &g) {
    return by_kind<Group>(h->prec, dt, h, s, g);
}

cudaError_t launch_bwd_prep(const Handle *h, cudaStream_t s, const void *x, plv_dtype dt,
                            int64_t rows, int log2T, int64_t ldx, float *P, float *rinv,
                            int T, const ConvPlan *plan, void *Ps, int N) {
    if (plan) {
        const K1Args a{x, ldx, P, rinv, N, T, 0, padded_len(T), rows, Ps};
        return dt == PLV_F32 ? k1_conv<float, kK1Prep>(h, s, a, *plan)
                             : k1_conv<double, kK1Prep>(h, s, a, *plan);
    }
    const K1Args a{x, ldx, P, rinv, N, T, log2T, (int64_t)1 << log2T, rows, Ps};
    return dt == PLV_F32 ? k1_pow2<float, kK1Prep>(h, s, a) : k1_pow2<double, kK1Prep>(h, s, a);
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
