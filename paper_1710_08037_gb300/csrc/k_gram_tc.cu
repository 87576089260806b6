// k_gram_tc.cu -- K3: the Hermitian Gram C = P P^H / T (Eq. 7) on the
// 5th-generation tensor cores (tcgen05), with the read-outs (Eq. 7, 13, 14)
// fused into the epilogue.
//
// Split precision.  Each phasor component p (Re or Im) is stored as two
// 16-bit numbers p = hi + lo (hi = RN(p), lo = RN(p - hi)), in BF16 or FP16.
// Every real product of the Gram is taken as hi*hi + hi*lo + lo*hi, the
// lo*lo term dropped, with FP32 accumulation in tensor memory.  With
// P = a + i b:
//     Re C = a a^T + b b^T,      Im C = b a^T - a b^T,
// so one K-block of samples costs 12 MMAs per output tile: 6 into the Re
// accumulator and 6 into the Im accumulator; the minus sign of a b^T is the
// MMA's negate-A bit.
//
// The same machinery serves the backward pass's dense contraction
// Gamma = S P / T (GEMM mode): A is the split rows of S (row i, K = k) and B
// P's own split rows (row k, t contiguous), which the MMA reads MN-major; with
// a, b the parts of S and a', b' those of P, Re Gamma = a a' - b b' and
// Im Gamma = b a' + a b' (12 MMAs again).  The tile grid is then full (every
// (I, J)) and the epilogue stores the complex tile instead of read-outs.
//
// Accumulation.  The tensor core's FP32 accumulation into TMEM does not
// round to nearest, and its error grows with the number of K blocks added
// into one accumulator.  So the K loop runs in chunks (1024 samples for
// BF16, 128 for FP16):
// each chunk accumulates into a fresh TMEM region (two regions, ping-pong),
// and the epilogue warps drain every finished chunk into FP32 running sums
// in registers (round to nearest), as a two-level summation.
//
// Kernel structure (one CTA per SM, persistent over the tile list):
//   warp 0      producer: per stage, one 32 KB bulk copy (cp.async.bulk)
//               per operand side -- the operand layout stores each block of
//               128 rows x 32 samples x 4 planes contiguously and already
//               64-byte swizzled -- into a 3-stage shared-memory ring;
//   warp 1      TMEM allocator and MMA issuer (one thread): tcgen05.mma
//               128x128x16, two TMEM regions of [128 Re + 128 Im] FP32
//               columns (512 columns) alternating per K chunk;
//   warps 2-17  epilogue: each owns one TMEM lane quarter (32 rows) and one
//               quarter of the columns (32), keeps 32 Re + 32 Im running
//               sums, drains each chunk, and at the end of the tile scales
//               by 1/T, applies the read-outs and stores the tile (vector
//               stores along rows) and its mirror (coalesced along columns).
// Only tiles (I, J) with I <= J of each epoch are computed; on a diagonal
// tile the B operand is the A operand already in shared memory.
//
// Work list.  A launch covers one problem (every epoch's upper-triangle
// tiles, enumerated in the kernel) or a group of problems of different N
// and T (an explicit list of (problem, epoch, I, J) items, longest first).
// CTAs take items round-robin; all three roles walk the same sequence.  In
// a group, a long tile may run as several split-K parts (whole chunks each)
// on different CTAs: each part stores its running sums in a slot, and per
// 32 x 32 block the last part to arrive (an atomic count, no waiting) adds
// the slots in part order and does the block's epilogue.
//
// Every wait on an mbarrier is bounded in time; on expiry the CTA records
// PLV_ERR_TIMEOUT in the device status word, stops issuing work, lets the
// copies and MMAs it issued land, frees its TMEM and returns.
#include "epilogue.cuh"

namespace plv {
namespace {

constexpr int TM = 128;                       // tile rows (i)
constexpr int TN = 128;                       // tile columns (j)
constexpr int KB = 32;                        // samples per stage
constexpr int NSTAGE = 3;
constexpr int PLANE_BYTES = TM * KB * 2;      // one 128 x 32 16-bit plane
constexpr int SIDE_BYTES = 4 * PLANE_BYTES;   // Re_hi, Re_lo, Im_hi, Im_lo
constexpr int STAGE_BYTES = 2 * SIDE_BYTES;   // A side + B side
constexpr int NEPI_WARPS = 16;               // 4 lane quarters x 4 column quarters
constexpr int NTHREADS = 64 + 32 * NEPI_WARPS;
constexpr int TMEM_COLS = 512;
constexpr int ACC_COLS = 256;                 // Re (128) + Im (128)
// Stages per K chunk, by split: BF16x3 drains every 1024 samples, FP16x3
// every 128.  Fewer drains made the N = T = 8192 Gram 6 % faster than 512
// (same-box A/B, under the power cap) but add accumulation error: the
// largest PLV error against the FP64 oracle there (on the diagonal, where
// the accumulators are largest) went from 5.5e-6 to 9.1e-6, within the
// BF16x3 bound of 2e-5.  The FP16 split is the accuracy-first mode.
template <uint32_t FMT>
struct Chunk {
    static constexpr int CH = FMT == 1u ? 32 : 4;
};
static_assert(Chunk<1u>::CH == 32 && Chunk<0u>::CH == 4, "gram_chunk_kb (common.cuh)");
static_assert(kTileFloats == 2 * TM * TN, "split-K chunk slot");
// per epilogue warp, a 32-row x 8-column FP32 staging tile for the row-wise
// stores (after the operand ring and the barriers)
constexpr int STAGE_TILE_FLOATS = 32 * 8;
constexpr int BAR_BYTES = 256;
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024 /*align*/ + BAR_BYTES +
                           NEPI_WARPS * STAGE_TILE_FLOATS * 4;
static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");

enum { P_RH = 0, P_RL = 1, P_IH = 2, P_IL = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- mbarrier -----------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase of parity `parity` completed; false on
// timeout (which raises the CTA's abort flag and the device status) or when
// another role already aborted.
__device__ __noinline__ bool wait_bar(uint32_t bar, uint32_t parity,
                                      volatile int *abort_flag, int *status,
                                      uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 127) == 0) {
            if (*abort_flag) return false;
            if (gtimer() - t0 > limit_ns) {
                *abort_flag = 1;
                atomicExch(status, (int)kDevTimeout);
                return false;
            }
        }
    }
}

// ---- bulk copy ---------------------------------------------------------------
// 1-D bulk copy global -> shared, completion counted on an mbarrier (16-byte
// aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"((uint64_t)src), "r"(bytes), "r"(bar)
        : "memory");
}

// ---- tcgen05 ------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     dst_smem),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The same MMA with the A operand kept in the tensor core's collector
// buffer: FILL reads A from shared memory and keeps it, USE takes the kept A
// (the same descriptor is passed), LAST takes it and releases the buffer.
// A group of MMAs sharing one A then reads it from shared memory once.  The
// MMAs of a group share one instruction descriptor: a group that mixed the
// negate bits gave wrong values on GB300 (measured), so the signs split the
// groups.
enum CollectorOp { kFill = 0, kUse = 1, kLast = 2 };
template <int OP>
__device__ __forceinline__ void mma_f16_ca(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate) {
    if constexpr (OP == kFill)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n\t}" ::"r"(
                d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else if constexpr (OP == kUse)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n\t}" ::"r"(
                d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}" ::"r"(
                d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            bar)
        : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
          "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
}
// Wait for this thread's tcgen05.ld results; the registers are in/out
// operands so no use of them can be scheduled above the wait.
__device__ __forceinline__ void tmem_ld_wait8(uint32_t (&a)[8], uint32_t (&b)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]),
                   "+r"(a[6]), "+r"(a[7]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]),
                   "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7])
                 :
                 : "memory");
}
// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, 8-row
// core-matrix groups 512 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
           ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// Shared-memory matrix descriptor: MN-major operand, 64-byte swizzle: atoms
// of 8 K-rows x 32 MN-elements (64 bytes each), the next 32 MN-elements
// 2048 bytes on (LBO), the next 8 K-rows 512 bytes on (SBO).
__device__ __forceinline__ uint64_t sdesc_mn64(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(2048 >> 4) << 16) |
           ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
constexpr uint32_t kIdescBMn = 1u << 16;  // instruction descriptor: B is MN-major

// Instruction descriptor, kind::f16: D = F32, A = B = BF16 (fmt 1) or FP16
// (fmt 0), both K-major, M = 128, N = 128, optional negate-A.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t fmt, bool negA, int n = TN) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((negA ? 1u : 0u) << 13) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// MMA width of a tile: its valid columns rounded up to 16 (the N step of an
// M = 128 MMA), so a ragged last column block costs only the columns it has.
// TMEM columns past it keep stale values, which no store reads.
__device__ __forceinline__ int mma_width(int valid) {
    return valid >= TN ? TN : ((valid + 15) & ~15);
}

struct TcArgs {
    TcProblem single;         // the problem when items == nullptr
    const TcProblem *probs;   // group: problem descriptors
    const int4 *items;        // group: (problem, epoch, I | J << 16, 1 + part or 0)
    TcSplit split;            // group: split-K parts of long tiles
    TcGemm gemm;              // GEMM mode: the contraction
    int total_items;
    int *status;
    uint64_t wait_ns;  // bound of every pipeline wait (the handle's wait limit)
    int stall;         // injected fault: each CTA withholds its first operand copy
};

// GEMM mode: item t is (epoch, I, J) with J fastest, so CTAs working at the
// same time share A row blocks and one epoch's B in L2.
__device__ __forceinline__ void gemm_item(const TcGemm &g, int t, int &e, int &I, int &J) {
    e = t / g.tpe;
    const int r = t - e * g.tpe;
    I = r / g.nrb_b;
    J = r - I * g.nrb_b;
}

// Item t: its problem, output matrix e, tile (I, J), K blocks [kb_lo,
// kb_hi) and split part (-1: the whole tile; always, unless SPLIT).
template <bool SPLIT>
__device__ __forceinline__ const TcProblem &item_of(const TcArgs &a, int t, int &e, int &I,
                                                    int &J, int &kb_lo, int &kb_hi, int &part) {
    if (a.items) {
        const int4 it = a.items[t];
        e = it.y;
        I = it.z & 0xffff;
        J = (int)((unsigned)it.z >> 16);
        const TcProblem &pb = a.probs[it.x];
        part = SPLIT ? it.w - 1 : -1;
        kb_lo = 0;
        kb_hi = pb.nkb;
        if (SPLIT && part >= 0) {
            const SplitPart &pr = a.split.parts[part];
            // checked builds: a part inside its tile's K range
            if (PLV_IN_BOUNDS(pr.kb_lo >= 0 && pr.kb_lo < pr.kb_hi && pr.kb_hi <= pb.nkb)) {
                kb_lo = pr.kb_lo;
                kb_hi = pr.kb_hi;
            }
        }
        return pb;
    }
    e = t / a.single.tpe;
    tile_raster(t - e * a.single.tpe, a.single.nrb, a.single.raster, I, J);
    kb_lo = 0;
    kb_hi = a.single.nkb;
    part = -1;
    return a.single;
}

// Split K, per 32 x 32 block of a tile: the warp stores its block of the
// part's sums in the part's slot and counts the arrival on the block's
// counter; the warp that completes the count (all S parts stored) adds the
// S slots in part order and returns true to store the block.  Writers fence
// before counting and the last one fences after, so it reads every part's
// slot (through L2, bypassing L1).
__device__ __forceinline__ bool split_last(const TcSplit &sp, const SplitPart &pr, int blk,
                                           int row, int cq, int lane, float (&sre)[32],
                                           float (&sim)[32]) {
    float *d = sp.partials + (size_t)pr.slot * kTileFloats + (size_t)row * TN + cq * 32;
#pragma unroll
    for (int k = 0; k < 32; k += 4) {
        __stcg((float4 *)(d + k), make_float4(sre[k], sre[k + 1], sre[k + 2], sre[k + 3]));
        __stcg((float4 *)(d + TM * TN + k),
               make_float4(sim[k], sim[k + 1], sim[k + 2], sim[k + 3]));
    }
    __threadfence();
    __syncwarp();
    int old = 0;
    if (lane == 0) old = atomicAdd(sp.counters + (size_t)pr.tile * 16 + blk, 1);
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old != pr.S - 1) return false;
    __threadfence();
    const float *b = sp.partials + (size_t)(pr.slot - pr.s) * kTileFloats + (size_t)row * TN +
                     cq * 32;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        sre[k] = 0.f;
        sim[k] = 0.f;
    }
    for (int r = 0; r < pr.S; ++r, b += kTileFloats) {
#pragma unroll
        for (int k = 0; k < 32; k += 4) {
            const float4 vr = __ldcg((const float4 *)(b + k));
            const float4 vi = __ldcg((const float4 *)(b + TM * TN + k));
            sre[k] += vr.x;
            sre[k + 1] += vr.y;
            sre[k + 2] += vr.z;
            sre[k + 3] += vr.w;
            sim[k] += vi.x;
            sim[k + 1] += vi.y;
            sim[k + 2] += vi.z;
            sim[k + 3] += vi.w;
        }
    }
    return true;
}

// SPLIT: the launch list holds split parts (grouped plans with split K);
// the other instantiations carry none of the split code.
template <uint32_t FMT, bool GEMM, bool SPLIT = false>
__global__ void __launch_bounds__(NTHREADS, 1)
k_gram_tc(const __grid_constant__ TcArgs args) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // stages, 1024-aligned
    uint8_t *gbase = smem_raw + (base - raw);
    uint64_t *bars = (uint64_t *)(gbase + NSTAGE * STAGE_BYTES);
    // bars: full[0..S), empty[0..S), tfull[2], tempty[2]
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * NSTAGE + 4);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    float *stage_tiles = (float *)(gbase + NSTAGE * STAGE_BYTES + BAR_BYTES);
    const uint32_t bar0 = smem_u32(bars);
    auto FULL = [&](int s) { return bar0 + 8u * s; };
    auto EMPTY = [&](int s) { return bar0 + 8u * (NSTAGE + s); };
    auto TFULL = [&](int b) { return bar0 + 8u * (2 * NSTAGE + b); };
    auto TEMPTY = [&](int b) { return bar0 + 8u * (2 * NSTAGE + 2 + b); };

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(FULL(s), 1);
            mbar_init(EMPTY(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(TFULL(b), 1);
            mbar_init(TEMPTY(b), 32 * NEPI_WARPS);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t pending = 0;        // stages with a copy issued
            uint32_t pend_parity = 0;    // FULL parity each pending copy completes
            // PLV_FAULT_STALL: the first stage is armed but its copies are
            // never issued, so the MMA issuer's wait for it runs into the bound
            bool withhold = args.stall != 0;
            for (int t = blockIdx.x; t < args.total_items && !*abort_flag; t += gridDim.x) {
                int e, I, J, nkb, kb_lo = 0, kb_hi;
                bool diag;
                const uint8_t *pa, *pj;
                if constexpr (GEMM) {
                    const TcGemm &g = args.gemm;
                    gemm_item(g, t, e, I, J);
                    diag = false;
                    nkb = g.nkb;
                    kb_hi = nkb;
                    pa = g.A + (size_t)((int64_t)e * g.nrb_a + I) * nkb * SIDE_BYTES;
                    // B: P's split blocks of epoch e, t-blocks 4J .. 4J + 3 of
                    // row block 0 (row block kb / 4 added per K block)
                    pj = g.B + (size_t)((int64_t)e * g.nrb_a * g.nkb_t + 4 * J) * SIDE_BYTES;
                    // checked builds: operand blocks inside both operands
                    if (!PLV_IN_BOUNDS(I >= 0 && I < g.nrb_a && J >= 0 && J < g.nrb_b &&
                                       4 * J < g.nkb_t && 4 * g.nrb_a >= nkb && e >= 0 &&
                                       (int64_t)e * g.tpe < args.total_items)) {
                        pa = g.A;
                        pj = g.B;
                    }
                } else {
                    int part;
                    const TcProblem &pb = item_of<SPLIT>(args, t, e, I, J, kb_lo, kb_hi, part);
                    diag = I == J;
                    nkb = pb.nkb;
                    // output matrix e: window w of epoch b
                    const int b = e / pb.nw, w = e - b * pb.nw;
                    const int64_t k0 = pb.kb0 + (int64_t)w * pb.hop_kb;
                    pa = pb.P + (size_t)(((int64_t)b * pb.nrb + I) * pb.kb_stride + k0) * SIDE_BYTES;
                    pj = pb.P + (size_t)(((int64_t)b * pb.nrb + J) * pb.kb_stride + k0) * SIDE_BYTES;
                    // checked builds: the tile's blocks inside its epoch's operand
                    if (!PLV_IN_BOUNDS(I >= 0 && I <= J && J < pb.nrb && e >= 0 && e < pb.batch &&
                                       k0 >= 0 && k0 + nkb <= pb.kb_stride)) {
                        pa = pb.P;
                        pj = pb.P;
                    }
                }
                for (int kb = kb_lo; kb < kb_hi; ++kb) {
                    if (!wait_bar(EMPTY(stage), phase ^ 1u, abort_flag, args.status, args.wait_ns)) break;
                    const uint32_t sa = base + stage * STAGE_BYTES;
                    // GEMM mode: B's t-blocks that exist (the last tile's
                    // others hold stale data, which only feeds columns t >= ld)
                    int nbv = 4;
                    if constexpr (GEMM)
                        nbv = args.gemm.nkb_t - 4 * J < 4 ? args.gemm.nkb_t - 4 * J : 4;
                    mbar_expect_tx(FULL(stage), diag ? SIDE_BYTES
                                                     : (GEMM ? SIDE_BYTES + nbv * SIDE_BYTES / 4
                                                             : 2 * SIDE_BYTES));
                    if (withhold) {
                        withhold = false;
                    } else {
                        bulk_g2s(sa, pa + (size_t)kb * SIDE_BYTES, SIDE_BYTES, FULL(stage));
                        if constexpr (GEMM) {
                            // rows k = 32 kb .. 32 kb + 31 of each t-block and
                            // plane (2 KB each) to [plane][t-block][32 rows]:
                            // the MN-major layout of the B descriptor
                            const uint8_t *src = pj +
                                                 (size_t)(kb >> 2) * args.gemm.nkb_t * SIDE_BYTES +
                                                 (size_t)(kb & 3) * (SIDE_BYTES / 16);
                            for (int c = 0; c < nbv; ++c)
                                for (int pl = 0; pl < 4; ++pl)
                                    bulk_g2s(sa + SIDE_BYTES + pl * PLANE_BYTES +
                                                 c * (PLANE_BYTES / 4),
                                             src + (size_t)c * SIDE_BYTES + pl * PLANE_BYTES,
                                             PLANE_BYTES / 4, FULL(stage));
                        } else if (!diag)
                            bulk_g2s(sa + SIDE_BYTES, pj + (size_t)kb * SIDE_BYTES, SIDE_BYTES,
                                     FULL(stage));
                        pending |= 1u << stage;
                        pend_parity = (pend_parity & ~(1u << stage)) | (phase << stage);
                    }
                    if (++stage == NSTAGE) { stage = 0; phase ^= 1u; }
                }
            }
            if (*abort_flag) {
                // let the copies already issued land before the CTA exits
                for (int st = 0; st < NSTAGE; ++st) {
                    if (!(pending & (1u << st))) continue;
                    const uint32_t par = (pend_parity >> st) & 1u;
                    const uint64_t t0 = gtimer();
                    while (!mbar_try_wait(FULL(st), par) && gtimer() - t0 < 100000000ull) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int buf = 0;
            uint32_t buf_phase = 0;
            bool issued = false;
            uint32_t last_bar = 0, last_parity = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < args.total_items && !*abort_flag;
                 t += gridDim.x) {
                int e, I, J, kb_lo = 0, kb_hi, ncols;
                bool diag;
                if constexpr (GEMM) {
                    gemm_item(args.gemm, t, e, I, J);
                    diag = false;
                    kb_hi = args.gemm.nkb;
                    ncols = (int)args.gemm.ld - J * TN;
                } else {
                    int part;
                    const TcProblem &pb = item_of<SPLIT>(args, t, e, I, J, kb_lo, kb_hi, part);
                    diag = I == J;
                    ncols = pb.N - J * TN;
                }
                const int nw = mma_width(ncols);
                const uint32_t ID_POS = idesc_f16(FMT, false, nw);
                const uint32_t ID_NEG = idesc_f16(FMT, true, nw);
                for (int kb0 = kb_lo; ok && kb0 < kb_hi; kb0 += Chunk<FMT>::CH) {
                    if (!wait_bar(TEMPTY(buf), buf_phase ^ 1u, abort_flag, args.status, args.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_re = tmem + buf * ACC_COLS;
                    const uint32_t d_im = d_re + TN;
                    const int kb1 = kb0 + Chunk<FMT>::CH < kb_hi ? kb0 + Chunk<FMT>::CH : kb_hi;
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!wait_bar(FULL(stage), phase, abort_flag, args.status, args.wait_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sa = base + stage * STAGE_BYTES;
                        const uint32_t sb = diag ? sa : sa + SIDE_BYTES;
                        if constexpr (GEMM) {
                            const uint32_t IP = ID_POS | kIdescBMn, IN = ID_NEG | kIdescBMn;
#pragma unroll
                            for (int ks = 0; ks < KB / 16; ++ks) {
                                const uint32_t ko = ks * 32;    // A: 16 K-values x 2 bytes
                                const uint32_t kr = ks * 1024;  // B: 16 K-rows x 64 bytes
                                const uint64_t aRH = sdesc_sw64(sa + P_RH * PLANE_BYTES + ko);
                                const uint64_t aRL = sdesc_sw64(sa + P_RL * PLANE_BYTES + ko);
                                const uint64_t aIH = sdesc_sw64(sa + P_IH * PLANE_BYTES + ko);
                                const uint64_t aIL = sdesc_sw64(sa + P_IL * PLANE_BYTES + ko);
                                const uint64_t bRH = sdesc_mn64(sb + P_RH * PLANE_BYTES + kr);
                                const uint64_t bRL = sdesc_mn64(sb + P_RL * PLANE_BYTES + kr);
                                const uint64_t bIH = sdesc_mn64(sb + P_IH * PLANE_BYTES + kr);
                                const uint64_t bIL = sdesc_mn64(sb + P_IL * PLANE_BYTES + kr);
                                const uint32_t first = (kb == kb0 && ks == 0) ? 0u : 1u;
                                // Re += a a' - b b', Im += b a' + a b' (hi*hi + hi*lo
                                // + lo*hi each), grouped by A operand and sign
                                mma_f16_ca<kFill>(d_re, aRH, bRH, IP, first);
                                mma_f16_ca<kUse>(d_re, aRH, bRL, IP, 1u);
                                mma_f16_ca<kUse>(d_im, aRH, bIH, IP, first);
                                mma_f16_ca<kLast>(d_im, aRH, bIL, IP, 1u);
                                mma_f16_ca<kFill>(d_re, aRL, bRH, IP, 1u);
                                mma_f16_ca<kLast>(d_im, aRL, bIH, IP, 1u);
                                mma_f16_ca<kFill>(d_re, aIH, bIH, IN, 1u);
                                mma_f16_ca<kLast>(d_re, aIH, bIL, IN, 1u);
                                mma_f16_ca<kFill>(d_im, aIH, bRH, IP, 1u);
                                mma_f16_ca<kLast>(d_im, aIH, bRL, IP, 1u);
                                mma_f16(d_re, aIL, bIH, IN, 1u);
                                mma_f16(d_im, aIL, bRH, IP, 1u);
                            }
                        } else {
#pragma unroll
                        for (int ks = 0; ks < KB / 16; ++ks) {
                            const uint32_t ko = ks * 32;  // 16 samples x 2 bytes
                            const uint64_t aRH = sdesc_sw64(sa + P_RH * PLANE_BYTES + ko);
                            const uint64_t aRL = sdesc_sw64(sa + P_RL * PLANE_BYTES + ko);
                            const uint64_t aIH = sdesc_sw64(sa + P_IH * PLANE_BYTES + ko);
                            const uint64_t aIL = sdesc_sw64(sa + P_IL * PLANE_BYTES + ko);
                            const uint64_t bRH = sdesc_sw64(sb + P_RH * PLANE_BYTES + ko);
                            const uint64_t bRL = sdesc_sw64(sb + P_RL * PLANE_BYTES + ko);
                            const uint64_t bIH = sdesc_sw64(sb + P_IH * PLANE_BYTES + ko);
                            const uint64_t bIL = sdesc_sw64(sb + P_IL * PLANE_BYTES + ko);
                            const uint32_t first = (kb == kb0 && ks == 0) ? 0u : 1u;
                            // Re C += a a^T + b b^T and Im C += b a^T - a b^T, each real
                            // product as hi*hi + hi*lo + lo*hi, ordered by A operand and
                            // sign so that the A planes of a group come from shared memory
                            // once (collector buffer): 6 A reads per 16 samples, not 12
                            mma_f16_ca<kFill>(d_re, aRH, bRH, ID_POS, first);
                            mma_f16_ca<kLast>(d_re, aRH, bRL, ID_POS, 1u);
                            mma_f16_ca<kFill>(d_im, aRH, bIH, ID_NEG, first);
                            mma_f16_ca<kLast>(d_im, aRH, bIL, ID_NEG, 1u);
                            mma_f16(d_re, aRL, bRH, ID_POS, 1u);
                            mma_f16(d_im, aRL, bIH, ID_NEG, 1u);
                            mma_f16_ca<kFill>(d_re, aIH, bIH, ID_POS, 1u);
                            mma_f16_ca<kUse>(d_re, aIH, bIL, ID_POS, 1u);
                            mma_f16_ca<kUse>(d_im, aIH, bRH, ID_POS, 1u);
                            mma_f16_ca<kLast>(d_im, aIH, bRL, ID_POS, 1u);
                            mma_f16_ca<kFill>(d_re, aIL, bIH, ID_POS, 1u);
                            mma_f16_ca<kLast>(d_im, aIL, bRH, ID_POS, 1u);
                        }
                        }
                        mma_commit(EMPTY(stage));  // frees the stage when done
                        issued = true;
                        last_bar = EMPTY(stage);
                        last_parity = phase;
                        if (++stage == NSTAGE) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    mma_commit(TFULL(buf));  // chunk ready for the epilogue
                    if (++buf == 2) { buf = 0; buf_phase ^= 1u; }
                }
            }
            if (*abort_flag && issued) {
                // let the MMAs already issued finish before TMEM is freed: the
                // last commit completes when every earlier MMA has
                const uint64_t t0 = gtimer();
                while (!mbar_try_wait(last_bar, last_parity) && gtimer() - t0 < 100000000ull) {
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;                // TMEM lane quarter of this warp
        const int cq = (warp - 2) >> 2;        // column quarter of this warp
        const int row = q * 32 + lane;         // tile row owned by this thread
        int buf = 0;
        uint32_t buf_phase = 0;
        bool ok = true;
        for (int t = blockIdx.x; ok && t < args.total_items; t += gridDim.x) {
            int e, I, J, nkb, kb_lo = 0, kb_hi, part = -1;
            const TcProblem *pbp = nullptr;
            if constexpr (GEMM) {
                gemm_item(args.gemm, t, e, I, J);
                nkb = args.gemm.nkb;
                kb_hi = nkb;
            } else {
                pbp = &item_of<SPLIT>(args, t, e, I, J, kb_lo, kb_hi, part);
                nkb = pbp->nkb;
            }
            if constexpr (!GEMM) {
                if (part < 0 && nkb <= Chunk<FMT>::CH) {
                    // The whole K range is one chunk (short windows, Grams over
                    // trials): stream the accumulators from TMEM eight columns
                    // at a time straight into the stores, instead of holding
                    // all 32 columns in registers, and release the buffer after
                    // the stores.  Same values as the running-sum path (its sums
                    // start from +0 and add this one chunk).
                    if (!wait_bar(TFULL(buf), buf_phase, abort_flag, args.status, args.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const TcProblem &pb = *pbp;
                    const int N = pb.N;
                    const int i = I * TM + row;
                    const int j0 = J * TN + cq * 32;
                    const bool above = I != J || q < cq;
                    const bool below = I == J && q > cq;
                    const bool staged = above && !pb.out.C && I * TM + q * 32 + 32 <= N &&
                                        j0 + 32 <= N;
                    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + buf * ACC_COLS +
                                        cq * 32;
                    if (!below) {
#pragma unroll 1
                        for (int h = 0; h < 4; ++h) {
                            uint32_t ur[8], ui[8];
                            tmem_ld8(tq + 8 * h, ur);
                            tmem_ld8(tq + TN + 8 * h, ui);
                            tmem_ld_wait8(ur, ui);
                            float re[8], im[8];
#pragma unroll
                            for (int c = 0; c < 8; ++c) {
                                re[c] = 0.f + __uint_as_float(ur[c]);
                                im[c] = 0.f + __uint_as_float(ui[c]);
                            }
                            if (staged) {
#pragma unroll
                                for (int m = 0; m < 3; ++m)
                                    store_block8(pb.out, m, (int64_t)e * N * N, N, I * TM + q * 32,
                                                 j0 + 8 * h, lane, re, im, pb.invT,
                                                 stage_tiles + (warp - 2) * STAGE_TILE_FLOATS,
                                                 pb.out.vec_ok);
                            } else {
                                store_tile_row<8>(pb.out, (int64_t)e * N * N, N, i, j0 + 8 * h,
                                                  I == J, re, im, pb.invT, pb.invT_d,
                                                  pb.out.diag ? pb.out.diag + e : nullptr);
                            }
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(TEMPTY(buf));
                    if (++buf == 2) { buf = 0; buf_phase ^= 1u; }
                    continue;
                }
            }
            float sre[32], sim[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) { sre[c] = 0.f; sim[c] = 0.f; }
            for (int kb0 = kb_lo; kb0 < kb_hi; kb0 += Chunk<FMT>::CH) {
                if (!wait_bar(TFULL(buf), buf_phase, abort_flag, args.status, args.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + buf * ACC_COLS +
                                    cq * 32;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    uint32_t ur[8], ui[8];
                    tmem_ld8(tq + 8 * h, ur);
                    tmem_ld8(tq + TN + 8 * h, ui);
                    tmem_ld_wait8(ur, ui);
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        sre[8 * h + c] += __uint_as_float(ur[c]);
                        sim[8 * h + c] += __uint_as_float(ui[c]);
                    }
                }
                tc_fence_before();
                mbar_arrive(TEMPTY(buf));
                if (++buf == 2) { buf = 0; buf_phase ^= 1u; }
            }
            if (!ok) break;
            if constexpr (SPLIT) {
                // a split part: blocks below a diagonal tile's diagonal store
                // nothing; the others go through the tile's slots
                if (part >= 0) {
                    if (I == J && q > cq) continue;
                    const SplitPart &pr = args.split.parts[part];
                    // checked builds: the part's slots and counter exist
                    if (!PLV_IN_BOUNDS(pr.s >= 0 && pr.s < pr.S && pr.slot - pr.s >= 0 &&
                                       pr.slot - pr.s + pr.S <= args.split.nslots &&
                                       pr.tile >= 0 && pr.tile < args.split.ntiles))
                        continue;
                    if (!split_last(args.split, pr, q * 4 + cq, row, cq, lane, sre, sim))
                        continue;
                }
            }
            const int i = I * TM + row;
            if constexpr (GEMM) {
                // the complex tile, scaled, as planar FP32 rows [e N + i][2][ld]
                const TcGemm &g = args.gemm;
                const int64_t t0 = (int64_t)J * TN + cq * 32;
                if (i < g.N && t0 < g.ld) {  // ld is a multiple of 32: all 32 or none
                    float *gr = g.G + ((int64_t)e * g.N + i) * 2 * g.ld + t0;
#pragma unroll
                    for (int c = 0; c < 32; c += 4) {
                        *(float4 *)(gr + c) = make_float4(sre[c] * g.invT, sre[c + 1] * g.invT,
                                                          sre[c + 2] * g.invT,
                                                          sre[c + 3] * g.invT);
                        *(float4 *)(gr + g.ld + c) =
                            make_float4(sim[c] * g.invT, sim[c + 1] * g.invT,
                                        sim[c + 2] * g.invT, sim[c + 3] * g.invT);
                    }
                }
            } else {
                const TcProblem &pb = *pbp;
                const int N = pb.N;
                const int j0 = J * TN + cq * 32;
                // checked builds: the output matrix and the tile exist
                if (!PLV_IN_BOUNDS(e >= 0 && e < pb.batch && I >= 0 && I <= J &&
                                   J * TN < N + TN - 1 && J < pb.nrb))
                    continue;
                // warp-uniform, per 32 x 32 block of the warp: blocks strictly
                // above the diagonal (every block of an off-diagonal tile; those
                // with q < cq of a diagonal tile) whose rows and columns are all
                // in range take the staged stores, without C; blocks strictly
                // below the diagonal of a diagonal tile store nothing (the
                // mirror of block (cq, q) writes them); the rest (the diagonal's
                // blocks, partial edge blocks, C) take the element path
                const bool above = I != J || q < cq;
                const bool below = I == J && q > cq;
                const bool staged = above && !pb.out.C && I * TM + q * 32 + 32 <= N &&
                                    j0 + 32 <= N;
                if (below) {
                    // nothing to store
                } else if (staged)
                    store_tile_staged(pb.out, (int64_t)e * N * N, N, I * TM + q * 32, j0, lane,
                                      sre, sim, pb.invT,
                                      stage_tiles + (warp - 2) * STAGE_TILE_FLOATS,
                                      pb.out.vec_ok);
                else
                    store_tile_row(pb.out, (int64_t)e * N * N, N, i, j0, I == J, sre, sim,
                                   pb.invT, pb.invT_d, pb.out.diag ? pb.out.diag + e : nullptr);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

}  // namespace

TcProblem make_tc_problem(const void *P, int batch, int N, int T, GramOut out) {
    TcProblem p;
    p.P = (const uint8_t *)P;
    p.batch = batch;
    p.N = N;
    p.nrb = (int)row_blocks(N);
    p.nkb = (int)(padded_len(T) / KB);
    p.tpe = p.nrb * (p.nrb + 1) / 2;
    p.kb_stride = p.nkb;
    p.nw = 1;
    p.kb0 = 0;
    p.hop_kb = 0;
    p.invT = 1.0f / (float)T;
    p.invT_d = 1.0 / (double)T;
    p.raster = kDefaultRaster;
    p.out = out;
    return p;
}

TcProblem make_tc_window_problem(const void *P, int batch, int N, int T, int t0, int W, int hop,
                                 int nw, GramOut out) {
    TcProblem p = make_tc_problem(P, batch, N, T, out);
    p.batch = batch * nw;
    p.nkb = W / KB;
    p.kb_stride = (int)(padded_len(T) / KB);
    p.nw = nw;
    p.kb0 = t0 / KB;
    p.hop_kb = hop / KB;
    p.invT = 1.0f / (float)W;
    p.invT_d = 1.0 / (double)W;
    return p;
}



static cudaError_t launch_tc(const Handle *h, cudaStream_t s, TcArgs a) {
    if (a.total_items <= 0) return cudaSuccess;
    a.stall = take_fault(PLV_FAULT_STALL) ? 1 : 0;
    const int grid = a.total_items < h->num_sms ? a.total_items : h->num_sms;
    const bool fp16 = h->prec == PLV_PREC_FP16X3;
    const bool split = a.items && a.split.ntiles > 0;
    auto kern = split ? (fp16 ? k_gram_tc<0u, false, true> : k_gram_tc<1u, false, true>)
                      : (fp16 ? k_gram_tc<0u, false> : k_gram_tc<1u, false>);
    static LaunchSetup ls16, ls_bf, ls16s, ls_bfs;
    int per_sm = 0;
    cudaError_t e = setup_once(split ? (fp16 ? ls16s : ls_bfs) : (fp16 ? ls16 : ls_bf), kern,
                               NTHREADS, SMEM_BYTES, per_sm);
    if (e != cudaSuccess) return e;
    kern<<<grid, NTHREADS, SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gram_tc_windows(const Handle *h, cudaStream_t s, const void *P, int batch,
                                   int N, int T, int t0, int W, int hop, int nw, GramOut out) {
    TcArgs a;
    a.split = TcSplit{};
    a.single = make_tc_window_problem(P, batch, N, T, t0, W, hop, nw, out);
    a.single.raster = h->gram_raster;
    a.probs = nullptr;
    a.items = nullptr;
    const int64_t total = (int64_t)a.single.tpe * a.single.batch;
    if (total > 0x7fffffff) return cudaErrorInvalidConfiguration;
    a.total_items = (int)total;
    a.status = h->status;
    a.wait_ns = h->wait_ns;
    a.stall = 0;
    return launch_tc(h, s, a);
}

cudaError_t launch_gemm_tc(const Handle *h, cudaStream_t s, const TcGemm &g, int batch) {
    TcArgs a;
    a.split = TcSplit{};
    a.single = TcProblem{};
    a.probs = nullptr;
    a.items = nullptr;
    a.gemm = g;
    const int64_t total = (int64_t)g.tpe * batch;
    if (total > 0x7fffffff) return cudaErrorInvalidConfiguration;
    a.total_items = (int)total;
    a.status = h->status;
    a.wait_ns = h->wait_ns;
    a.stall = 0;
    if (a.total_items <= 0) return cudaSuccess;
    a.stall = take_fault(PLV_FAULT_STALL) ? 1 : 0;
    const int grid = a.total_items < h->num_sms ? a.total_items : h->num_sms;
    // the BF16 split: gradients can exceed the FP16 range
    auto kern = k_gram_tc<1u, true>;
    static LaunchSetup ls;
    int per_sm = 0;
    cudaError_t e = setup_once(ls, kern, NTHREADS, SMEM_BYTES, per_sm);
    if (e != cudaSuccess) return e;
    kern<<<grid, NTHREADS, SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gram_tc(const Handle *h, cudaStream_t s, const void *P, int batch,
                           int N, int T, GramOut out) {
    TcArgs a;
    a.split = TcSplit{};
    a.single = make_tc_problem(P, batch, N, T, out);
    a.single.raster = h->gram_raster;
    a.probs = nullptr;
    a.items = nullptr;
    const int64_t total = (int64_t)a.single.tpe * batch;
    if (total > 0x7fffffff) return cudaErrorInvalidConfiguration;
    a.total_items = (int)total;
    a.status = h->status;
    a.wait_ns = h->wait_ns;
    a.stall = 0;
    return launch_tc(h, s, a);
}

static __global__ void k_zero_group_diag(const TcProblem *probs, int nprob) {
    for (int p = blockIdx.x; p < nprob; p += gridDim.x) {
        double *d = probs[p].out.diag;
        if (!d) continue;
        for (int e = threadIdx.x; e < probs[p].batch; e += blockDim.x) d[e] = 0.0;
    }
}

cudaError_t launch_zero_group_diag(cudaStream_t s, const TcProblem *probs, int nprob) {
    if (nprob <= 0) return cudaSuccess;
    k_zero_group_diag<<<nprob < 1024 ? nprob : 1024, 128, 0, s>>>(probs, nprob);
    return cudaGetLastError();
}

cudaError_t launch_gram_tc_group(const Handle *h, cudaStream_t s, const TcProblem *probs,
                                 const int4 *items, int nitems, const TcSplit &split) {
    TcArgs a;
    a.single = TcProblem{};
    a.probs = probs;
    a.items = items;
    a.split = split;
    a.total_items = nitems;
    a.status = h->status;
    a.wait_ns = h->wait_ns;
    a.stall = 0;
    return launch_tc(h, s, a);
}

}  // namespace plv
