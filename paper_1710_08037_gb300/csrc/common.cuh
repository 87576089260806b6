// common.cuh -- internal declarations shared by the library's translation
// units: the handle, status helpers, the operand layouts and the kernel
// launchers.  Nothing here is part of the public ABI (include/plv.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <cmath>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "plv.h"

namespace plv {

// NVTX range around one entry point (header-only NVTX 3: a no-op unless a
// profiler attaches).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define PLV_RANGE(name) ::plv::NvtxRange plv_nvtx_range_(name)

// Checked builds (-DPLV_CHECKED=1).  PLV_IN_BOUNDS(c) guards an access by the
// bounds condition c of its index computation: true when c holds; when it
// fails, the access is skipped (the macro is false) and the source line is
// recorded in this translation unit's device word (the first failure wins),
// which plv_check_status reads.  Unchecked builds compile the condition away.
#ifndef PLV_CHECKED
#define PLV_CHECKED 0
#endif
typedef int (*CheckReader)();  // reads and clears one unit's word (current device)
int register_check_unit(CheckReader r);
#if PLV_CHECKED
// one word per translation unit: the library is linked without relocatable
// device code, so every unit records into its own
static __device__ int plv_check_line_;
#define PLV_IN_BOUNDS(c) \
    ((c) ? true : (atomicCAS(&plv_check_line_, 0, (int)__LINE__), false))
static int plv_check_read_() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, plv_check_line_, sizeof(int)) != cudaSuccess) return 0;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(plv_check_line_, &z, sizeof(int));
    }
    return v;
}
static const int plv_check_registered_ = register_check_unit(&plv_check_read_);
#else
#define PLV_IN_BOUNDS(c) true
#endif

// Phasor operand rows are padded to a multiple of this many samples (the
// Gram's K tile); the padding holds zeros.
constexpr int kPadT = 32;

__host__ __device__ inline int64_t padded_len(int T) {
    return ((int64_t)T + kPadT - 1) / kPadT * kPadT;
}

// Split-precision operand layout (BF16X3 / FP16X3): blocks of 128 rows x 32
// samples x 4 planes (Re_hi, Re_lo, Im_hi, Im_lo) of 16-bit values, 32 KB
// each, contiguous and already in the tensor-core shared-memory layout
// (K-major, 64-byte rows, 64-byte swizzle: the 16-byte chunk c of row r sits
// at chunk c ^ ((r >> 1) & 3)).  Block (e, rb, kb) starts at
// ((e * NRB + rb) * NKB + kb) * 32 KB with NRB = ceil(N / 128) row blocks and
// NKB = ld / 32 sample blocks.  Rows N .. NRB*128-1 and samples T .. ld-1
// are zero.
constexpr int kTileRows = 128;
constexpr int kTileK = 32;
constexpr int kBlockElems = 4 * kTileRows * kTileK;  // 16-bit elements per block
__host__ __device__ inline int64_t row_blocks(int N) { return ((int64_t)N + kTileRows - 1) / kTileRows; }

__host__ __device__ inline int64_t split_offset(int64_t e, int64_t n, int64_t t, int64_t NRB,
                                                int64_t NKB) {
    const int64_t rb = n >> 7, r = n & 127, kb = t >> 5, k = t & 31;
    const int64_t blk = (e * NRB + rb) * NKB + kb;
    const int64_t kc = ((((k >> 3) ^ ((r >> 1) & 3)) << 3) | (k & 7));
    return blk * kBlockElems + r * kTileK + kc;  // plane 0; plane p at + p * 4096
}

// Smallest and largest power-of-two lengths the shared-memory FFT handles.
constexpr int kMinLog2T = 5;
constexpr int kMaxLog2T = 14;        // twiddle tables
constexpr int kMaxLog2Direct = 13;   // lengths the two-buffer FFT kernel fits
constexpr int kMinLog2Bands = 7;     // shortest length of the multi-band transform

// Device status codes written by kernels into the handle's status word.
enum : int { kDevOk = 0, kDevTimeout = 5 };

// Plan of the any-length Hilbert transform (fft.cuh): FFT length M and its
// decimation-in-frequency radix order, twiddles exp(-2 pi i m / M), and the
// Hilbert kernel's spectrum factor S / M in that transform's output order.
struct ConvPlan {
    int M;
    int nstages;
    int radix[8];
    const float2 *tw;
    const float *S;
};
constexpr int kMaxConvM = 24576;  // 3 * 2^13: T up to 12288
// Thread classes of the any-length engine: CTAs of kConvThreads[c] threads
// take transform lengths M <= kConvMaxM[c].  As many CTAs per SM as the
// shared buffer allows (each CTA is its own barrier domain), with the SM's
// register file split among them at kConvRegs registers per thread.  Radix
// stages are at most kConvMaxRadix.
constexpr int kConvClasses = 4;
constexpr int kConvRegs = 64;
constexpr int kConvMaxRadix = 8;
__host__ __device__ constexpr int conv_class_threads(int c) {
    return c == 0 ? 128 : c == 1 ? 256 : c == 2 ? 512 : 1024;
}
__host__ __device__ constexpr int conv_class_max_M(int c) {
    return c == 0 ? 3072 : c == 1 ? 6144 : c == 2 ? 12288 : kMaxConvM;
}
__host__ __device__ constexpr int conv_class(int M) {
    return M <= conv_class_max_M(0) ? 0 : M <= conv_class_max_M(1) ? 1
         : M <= conv_class_max_M(2) ? 2 : 3;
}
__host__ __device__ constexpr int conv_threads(int M) {
    return conv_class_threads(conv_class(M));
}
__host__ __device__ constexpr size_t conv_smem(int M) {
    return (size_t)(M + M / 32) * sizeof(float2);
}
// Persistent CTAs of one any-length launch of transform length M (the
// occupancy the class's register budget allows, on every SM).
inline int64_t conv_grid(int num_sms, int M) {
    const int per_sm = 65536 / (kConvRegs * conv_class_threads(conv_class(M)));
    return (int64_t)(per_sm > 0 ? per_sm : 1) * num_sms;
}

// Orders of the grouped Gram's tile list.  The persistent launch hands item
// t to CTA t mod G (G = its grid), so an order is a schedule.
enum GramSchedule : int {
    kSchedLongestFirst = 0,  // by K blocks, descending (plan default)
    kSchedBalanced = 1,      // longest first, each round of G items dealt to
                             // the least-loaded CTAs (greedy LPT per round)
};

// Launch configuration of a plan, as chosen by the autotuner (defaults:
// every transform length in its own thread class, occupancy-limited grids,
// longest-first tiles).
struct GroupConfig {
    std::map<int, int> k1_class;        // transform length M -> thread class
    int k1_per_sm[kConvClasses] = {0, 0, 0, 0};  // 0: occupancy limit
    int gram_schedule = kSchedLongestFirst;
    int gram_tile_cost = 0;             // per-tile fixed cost, in K blocks
    int gram_split = 0;                 // split-K factor f (0: no tile split)
    bool operator==(const GroupConfig &o) const {
        for (int c = 0; c < kConvClasses; ++c)
            if (k1_per_sm[c] != o.k1_per_sm[c]) return false;
        return k1_class == o.k1_class && gram_schedule == o.gram_schedule &&
               gram_tile_cost == o.gram_tile_cost && gram_split == o.gram_split;
    }
};

// Tile t of the column-major upper triangle: t = J (J + 1) / 2 + I, I <= J.
__host__ __device__ inline void upper_tile_of(int t, int &I, int &J) {
    int j = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((j + 1) * (j + 2) / 2 <= t) ++j;
    while (j * (j + 1) / 2 > t) --j;
    J = j;
    I = t - j * (j + 1) / 2;
}

// Tile order of a single problem's epoch (the tensor-core Gram, k_gram_tc.cu).  The persistent CTAs take items
// round-robin, so G consecutive items (G = the grid) run at about the same
// time and stream their row panels through L2 together; an order whose G
// consecutive tiles touch few distinct row blocks re-reads fewer panels from
// DRAM.  Tiles go by super-columns of W block columns; in each, the
// off-diagonal super-blocks (W rows x wj columns, column-major), then the
// diagonal super-block's triangle (column-major).  With nrb <= W this is the
// plain column-major triangle.  (A lockstep model of N = 8192, 152 CTAs:
// 431 panel reads per epoch at W = 16 against 639 for the column-major
// triangle.)  The order changes which CTA computes a tile, never its value.
__host__ __device__ inline void tile_raster(int t, int nrb, int W, int &I, int &J) {
    int SJ = 0, wj = nrb < W ? nrb : W;
    for (;;) {
        const int cnt = SJ * W * wj + wj * (wj + 1) / 2;  // tiles of super-column SJ
        if (t < cnt) break;
        t -= cnt;
        ++SJ;
        wj = nrb - SJ * W < W ? nrb - SJ * W : W;
    }
    const int offd = SJ * W * wj;
    if (t < offd) {
        const int SI = t / (W * wj);
        const int r = t - SI * W * wj;
        const int jj = r / W;
        I = SI * W + (r - jj * W);
        J = SJ * W + jj;
    } else {
        int ii, jj;
        upper_tile_of(t - offd, ii, jj);
        I = SJ * W + ii;
        J = SJ * W + jj;
    }
}

// Default raster width of the single-problem Gram's tile order (k_gram_tc.cu).
constexpr int kDefaultRaster = 8;
// Default bound of every wait of the tensor-core Gram's pipeline (4 s).  The
// clean-up waits of an aborting CTA keep their own fixed bound (0.1 s).
constexpr uint64_t kDefaultWaitNs = 4000000000ull;

struct Handle {
    int device = 0;
    int gram_raster = kDefaultRaster;  // tile raster width of single-problem Grams
    uint64_t wait_ns = kDefaultWaitNs;  // pipeline wait bound of the tensor-core Gram
    plv_precision prec = PLV_PREC_FP32;
    size_t workspace_limit = 0;
    size_t workspace_used = 0;  // device bytes the handle holds now
    size_t workspace_peak = 0;  // and at most so far (plv_memory_usage)
    int num_sms = 0;
    // twiddles exp(-2 pi i m / 2^L), m < 2^L, for L = kMinLog2T..kMaxLog2T,
    // table L starting at element (2^L - 2^kMinLog2T)
    float2 *twiddles = nullptr;
    int *status = nullptr;  // device status word
    void *ws = nullptr;     // scratch for the backward pass (grows on demand)
    size_t ws_bytes = 0;
    // a stream capture used ws, so a graph may still hold its address: on
    // growth it is kept (retired) until plv_destroy rather than freed
    bool ws_in_graph = false;
    std::vector<void *> ws_retired;
    std::map<int, ConvPlan> conv;      // by T (lengths that are not handled directly)
    std::map<int, float2 *> conv_tw;   // twiddle tables by M
    std::map<int, float *> conv_S;     // kernel spectra by T
    // band-limited analytic-signal kernel spectra ([nbands][M] complex), by a
    // hash of (T, nbands, mask values)
    std::map<uint64_t, float2 *> band_K;
    // autotuned configurations of grouped plans, by the plan's work signature
    std::map<std::string, GroupConfig> tuned;
    std::mutex mu;
};

// Record a new value of h.workspace_used in the high-water mark.
inline void note_usage(Handle &h) {
    if (h.workspace_used > h.workspace_peak) h.workspace_peak = h.workspace_used;
}

// Per-kernel launch set-up done once per device (the shared-memory opt-in
// and the occupancy query are not stream operations, and doing them once
// keeps later launches free of them, e.g. inside a graph capture).
struct LaunchSetup {
    int per_sm[64] = {0};  // 0: not set up yet on that device
};
template <typename Kern>
inline cudaError_t setup_once(LaunchSetup &ls, Kern kern, int threads, size_t smem,
                              int &per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (ls.per_sm[dev] == 0) {
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return e;
        }
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem);
        if (e != cudaSuccess) return e;
        ls.per_sm[dev] = n > 0 ? n : 1;
    }
    per_sm = ls.per_sm[dev];
    return cudaSuccess;
}

// The any-length plan for T (built and cached on first use: allocates).
plv_status get_conv_plan(Handle &h, int T, const ConvPlan **plan);
// The any-length plan for T plus, for each of the nbands device masks
// [nbands][T/2 + 1], the spectrum K_b (divided by M, in the transform's
// output order) of the band-limited analytic-signal kernel IDFT_T(h B_b):
// reads the masks back (synchronises s), cached by their values.
plv_status get_band_plan(Handle &h, cudaStream_t s, int T, const float *masks, int nbands,
                         const ConvPlan **plan, const float2 **K);
void free_conv_plans(Handle &h);
// The multi-band analytic signal for T = 2^log2T (k_bands.cu): nbands
// operand buffers band_bytes apart.
cudaError_t launch_analytic_bands(const Handle *h, cudaStream_t s, const void *x, plv_dtype dt,
                                  int64_t rows, int N, int log2T, int64_t ldx, const float *masks,
                                  int nbands, void *P, int64_t band_bytes);
// The multi-band analytic signal for lengths other than the power-of-two
// band kernel's: one row per transform, the spectrum kept in scratch
// (conv_grid(num_sms, M) slots of M complex values), nbands kernel spectra K.
cudaError_t launch_analytic_bands_conv(const Handle *h, cudaStream_t s, const void *x,
                                       plv_dtype dt, int64_t rows, int N, int T, int64_t ldx,
                                       const ConvPlan &plan, const float2 *K, int nbands,
                                       void *P, int64_t band_bytes, float2 *scratch);
// K1 for lengths the direct FFT does not take (any T up to kMaxConvM / 2).
cudaError_t launch_analytic_conv(const Handle *h, cudaStream_t s, const void *x,
                                 plv_dtype dt, int64_t rows, int N, int T, int64_t ldx,
                                 void *P, const ConvPlan &plan);

// One problem of a grouped K1 launch (device descriptor; words copied to
// shared memory by the kernel, so the size is a multiple of 4 bytes).
struct K1Desc {
    const void *x;
    void *P;
    int64_t ldx, ld, rows;  // x row stride, phasor row length, batch * N
    int N, T;
    ConvPlan plan;
};
// A grouped K1 plan: every (problem, row pair) of the group, by thread class
// (conv_class) and within a class by decreasing M.
struct K1Group {
    const K1Desc *descs;     // device
    const int2 *items;       // device: (problem, row pair)
    int64_t begin[kConvClasses], count[kConvClasses];
    int max_M[kConvClasses];
    int per_sm[kConvClasses];  // CTAs per SM of each class launch; 0: occupancy limit
};
// K1 of every problem of a group: one persistent launch per non-empty class.
cudaError_t launch_analytic_group(const Handle *h, cudaStream_t s, plv_dtype dt,
                                  const K1Group &g);

// Per-thread last error message.
void set_error(const char *fmt, ...);
plv_status fail(plv_status s, const char *fmt, ...);
plv_status check_cuda(cudaError_t e, const char *what);
// As check_cuda for a device allocation: PLV_ERR_ALLOC on failure.
plv_status check_alloc(cudaError_t e, const char *what);

// Host-side fault injection (plv_debug_fault, env PLV_FAULT): true when the
// armed fault is of `kind` and this event is the one it counts down to
// (which disarms it).
bool take_fault(int kind);
// cudaMalloc through the allocation fault hook.
cudaError_t dev_malloc_raw(void **p, size_t bytes);
template <class T>
inline cudaError_t dev_malloc(T **p, size_t bytes) {
    void *v = nullptr;
    const cudaError_t e = dev_malloc_raw(&v, bytes);
    *p = (T *)v;
    return e;
}
// check_cuda of a kernel launch through the launch fault hook: an injected
// fault returns PLV_ERR_CUDA without evaluating (launching) `expr`.
#define PLV_CHECK_LAUNCH(expr, what)                                                      \
    (::plv::take_fault(PLV_FAULT_LAUNCH)                                                  \
         ? ::plv::fail(PLV_ERR_CUDA, "%s: injected launch failure", (what))              \
         : ::plv::check_cuda((expr), (what)))

inline const float2 *twiddle_table(const Handle *h, int log2T) {
    return h->twiddles + ((1 << log2T) - (1 << kMinLog2T));
}

// ---- kernel launchers (one translation unit each) --------------------------

// K1: fused Hilbert FFT + normalisation, power-of-two T.
cudaError_t launch_analytic_pow2(const Handle *h, cudaStream_t s,
                                 const void *x, plv_dtype dt, int64_t rows,
                                 int N, int log2T, int64_t ldx, void *P);
// Zero the padding rows N .. NRB*128-1 of a split-precision phasor buffer.
cudaError_t launch_zero_pad_rows(cudaStream_t s, void *P, int batch, int N, int T);
// Backward preparation: FP32 phasors P[rows][2][ld] and rinv[rows][ld]; with
// Ps, P also as BF16 splits in the tiled operand layout (rows of N per epoch).
cudaError_t launch_bwd_prep(const Handle *h, cudaStream_t s, const void *x, plv_dtype dt,
                            int64_t rows, int log2T, int64_t ldx, float *P, float *rinv,
                            int T, const ConvPlan *plan, void *Ps = nullptr, int N = 0);
// K5: S = G + G^H, Gamma = S P / T, grad = Re Gamma_z - H{Im Gamma_z}.
// tc_a NULL: FP32 contraction on the CUDA cores with S FP32 planar
// [batch][2][N][N]; else the tensor-core contraction, with S written as
// split rows at tc_a (the first a_bytes of backward_tc_bytes) and tc_b P's
// BF16 split rows in the operand layout (the preparation wrote them), S unused.
cudaError_t launch_backward(const Handle *h, cudaStream_t st, int batch, int N, int T,
                            int log2T, const float2 *C, const float *g1, const float *g2,
                            const float *g3, const float *P, const float *rinv, float *S,
                            float *Gm, float *grad, const ConvPlan *plan, void *tc_a,
                            const void *tc_b);
// Bytes of the tensor-core backward's split operands (S rows, then P's split
// rows); *a_bytes receives the first part's size.
size_t backward_tc_bytes(int batch, int N, int T, size_t *a_bytes);
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
// One problem of a grouped tensor-core launch (device descriptor): phasors
// in the tiled split layout, sizes and outputs.
struct TcProblem {
    const uint8_t *P;
    int batch, N, nrb, nkb, tpe;  // output matrices, rows, row blocks, K blocks, tiles/matrix
    // sample windows: output matrix e is window w = e % nw of epoch e / nw and
    // covers K blocks kb0 + w * hop_kb .. + nkb of rows kb_stride blocks long
    // (one window, kb_stride = nkb and kb0 = 0, for the whole epoch)
    int kb_stride, nw, kb0, hop_kb;
    float invT;
    double invT_d;
    int raster;  // tile raster width in row blocks (single-problem launches)
    GramOut out;
};
TcProblem make_tc_problem(const void *P, int batch, int N, int T, GramOut out);
// Sliding windows of W samples (t0, W, hop multiples of 32) over each epoch.
TcProblem make_tc_window_problem(const void *P, int batch, int N, int T, int t0, int W, int hop,
                                 int nw, GramOut out);
cudaError_t launch_gram_tc_windows(const Handle *h, cudaStream_t s, const void *P, int batch,
                                   int N, int T, int t0, int W, int hop, int nw, GramOut out);
cudaError_t launch_gram_fp32_windows(const Handle *h, cudaStream_t s, const float *P, int batch,
                                     int N, int T, int t0, int W, int hop, int nw, GramOut out);
// The backward pass's contraction on the tensor cores (BF16 split):
// G[e][i][2][ld] = (1/T) sum_k S[e][i][k] P[e][k][t], from A = split rows of S
// (row i, K = k; rows padded to nrb_a blocks of 128, nkb blocks of 32 along
// k) and B = P's own split rows (row k, t contiguous: nrb_a blocks of 128
// rows, nkb_t blocks of 32 along t), read by the MMA as an MN-major operand.
// Tiles (I, J) of 128 rows i x 128 samples t, nrb_b = ceil(ld / 128) along t,
// every tile of every epoch.
struct TcGemm {
    const uint8_t *A, *B;
    int nrb_a, nrb_b, nkb, tpe;  // tpe = nrb_a * nrb_b tiles per epoch
    int nkb_t;                   // 32-sample blocks along t of B's layout (ld / 32)
    int N;                       // valid rows i (and k)
    int64_t ld;                  // row length of G (valid t)
    float invT;
    float *G;
};
cudaError_t launch_gemm_tc(const Handle *h, cudaStream_t s, const TcGemm &g, int batch);
// Split K of a grouped Gram.  A long tile may run as S parts, each over a
// range of whole K chunks (the chunks of the two-level summation), on
// different CTAs.  A part adds its chunks' sums as an unsplit tile does and
// stores the result in its slot of `partials`; per 32 x 32 block of the
// tile, the warp that completes the block's count of S arrivals adds the S
// slots in part order (a fixed order: every run gives the same bits) and
// stores the block.
struct SplitPart {
    int kb_lo, kb_hi;  // K blocks of the part
    int tile;          // the tile's counter index
    int slot;          // this part's slot; the tile's parts use slot - s .. + S - 1
    int s, S;          // part s of S
    int pad[2];
};
struct TcSplit {
    const SplitPart *parts = nullptr;
    float *partials = nullptr;  // [slot][Re, Im][128][128] FP32
    int *counters = nullptr;    // [split tile][16 blocks], zero before each launch
    int nslots = 0, ntiles = 0; // sizes of partials (slots) and counters (tiles)
};
constexpr int kTileFloats = 2 * 128 * 128;  // one slot
// K blocks of 32 samples per chunk of the two-level summation (BF16x3: 1024
// samples, FP16x3: 128).
inline int gram_chunk_kb(plv_precision p) { return p == PLV_PREC_FP16X3 ? 4 : 32; }
// One persistent launch over a list of tiles: items[t] = (problem, epoch,
// I | J << 16, 1 + split part, or 0 for a whole tile).
cudaError_t launch_gram_tc_group(const Handle *h, cudaStream_t s, const TcProblem *probs,
                                 const int4 *items, int nitems, const TcSplit &split);
// Zero the diagonal-check outputs of every problem of a group.
cudaError_t launch_zero_group_diag(cudaStream_t s, const TcProblem *probs, int nprob);
// Operands of a Gram over trials (k_trials.cu): one problem per column.
cudaError_t launch_trial_operands(const Handle *h, cudaStream_t s, const float *V, int E, int N,
                                  int64_t ldv, int l0, int L, int rms, void *P);
// DFT of real rows at selected bins (k_dft.cu), FP32 planar rows out.
cudaError_t launch_dft_bins(cudaStream_t s, const void *x, plv_dtype dt, int64_t rows, int T,
                            int64_t ldx, int f0, int F, float *X, int64_t ldX);
// K6: read-outs from a stored C.
cudaError_t launch_metrics(cudaStream_t s, const float2 *C, int batch, int N,
                           float *plv, float *iplv, float *ciplv);

}  // namespace plv

struct plv_handle {
    plv::Handle h;
};
