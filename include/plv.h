/*
 * plv.h -- C ABI of the GB300 Phase Locking Value library.
 *
 * Computes, for every epoch of real band-limited signals x (N channels x T
 * samples), the time-averaged phase locking value of Bruna, Maestu & Pereda,
 * "Phase Locking Value revisited", in its reformulated form:
 *
 *   z   = x + i H{x}                 analytic signal            (Eq. 3)
 *   P   = z / |z|                    unit phasors               (Eq. 4)
 *   C   = P P^H / T                  Hermitian Gram             (Eq. 5-7)
 *   PLV = |C|, iPLV = |Im C|,                                   (Eq. 7, 13)
 *   ciPLV = Im C / sqrt((1 - Re C)(1 + Re C))                   (Eq. 14)
 *
 * Conventions shared by every entry point
 *   - All data pointers are DEVICE pointers unless stated otherwise, owned by
 *     the caller; the library never frees them.  The handle owns its own
 *     workspace (twiddle tables, a device status word, backward scratch).
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Every call is asynchronous on that stream.
 *   - Arguments are validated on the host before anything is launched; a
 *     validation failure returns PLV_ERR_INVALID (or PLV_ERR_UNSUPPORTED for
 *     a valid but unimplemented shape) and launches nothing.
 *   - Device-side failures (a bounded wait that gave up) are recorded in the
 *     handle's device status word; plv_sync_status() reads and clears it.
 *   - plv_last_error() returns a message for the last failing call made on
 *     the calling thread; the string is owned by the library.
 *   - Sign convention: C_ij = (1/T) sum_t P_i(t) conj(P_j(t)), so Im C_ij > 0
 *     (and ciPLV_ij > 0) when channel i leads channel j.
 *   - Readings where the paper is silent: a sample with |z| = 0 has P = 0 and
 *     contributes nothing; ciPLV = 0 where (1 - Re C)(1 + Re C) <= 0; the
 *     diagonal of iPLV and ciPLV is 0; the analytic signal is the periodic
 *     discrete one over exactly the T samples given (no padding inside).
 *   - Outputs are full N x N squares per epoch: the upper triangle is
 *     computed and mirrored (PLV, iPLV symmetric; ciPLV antisymmetric, bit
 *     for bit).
 */
#ifndef PLV_H
#define PLV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct plv_handle plv_handle;

typedef enum {
    PLV_OK = 0,
    PLV_ERR_INVALID = 1,     /* bad argument: null pointer, negative size... */
    PLV_ERR_ALLOC = 2,       /* device or host allocation failed            */
    PLV_ERR_CUDA = 3,        /* a CUDA runtime call failed                  */
    PLV_ERR_UNSUPPORTED = 4, /* valid request this build does not implement */
    PLV_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up          */
    PLV_ERR_NUMERIC = 6      /* reserved: non-finite data in checked mode   */
} plv_status;

typedef enum { PLV_F32 = 0, PLV_F64 = 1 } plv_dtype;

/* Arithmetic of the Gram (Eq. 7).  FP32: FP32 phasors, FP32 FMA on the CUDA
 * cores.  BF16X3: each phasor component split as hi + lo, two BF16 numbers;
 * the Gram is hi*hi + hi*lo + lo*hi on the tensor cores (tcgen05) with FP32
 * accumulation.  FP16X3: the same with FP16 hi + lo (11-bit significands,
 * so the split carries 22 bits instead of 16; same tensor-core rate). */
typedef enum {
    PLV_PREC_FP32 = 0,
    PLV_PREC_BF16X3 = 1,
    PLV_PREC_FP16X3 = 2
} plv_precision;

enum {
    PLV_OUT_PLV = 1,   /* |C|                         (Eq. 7)  */
    PLV_OUT_IPLV = 2,  /* |Im C|                      (Eq. 13) */
    PLV_OUT_CIPLV = 4, /* Im C / sqrt(1 - (Re C)^2)   (Eq. 14) */
    PLV_OUT_C = 8      /* C itself, complex64 interleaved      */
};

/* Create a handle bound to CUDA device `device` with Gram arithmetic `prec`.
 * `workspace_limit` caps the handle's device workspace in bytes (0 = no
 * cap).  Allocates (cudaMalloc) -- call outside stream capture.
 * Errors: PLV_ERR_INVALID (h NULL, bad device or precision), PLV_ERR_CUDA,
 * PLV_ERR_ALLOC. */
plv_status plv_create(plv_handle **h, int device, plv_precision prec,
                      size_t workspace_limit);

/* Destroy a handle and free its workspace (synchronises the device).  NULL
 * is accepted and ignored. */
plv_status plv_destroy(plv_handle *h);

/* Message for the last failing call on this thread ("" if none). */
const char *plv_last_error(const plv_handle *h);

/* Gram arithmetic the handle was created with. */
plv_precision plv_get_precision(const plv_handle *h);

/* Tile order of the tensor-core Gram of later plv_gram / plv_gram_windows
 * calls on this handle (no counterpart in the paper: a schedule of the
 * Eq. 7 tiles, which changes which CTA computes a tile, never its value).
 * The 128 x 128 upper-triangle tiles of each epoch go by super-columns of
 * `width` 128-row blocks, so that the tiles running at the same time share
 * their row panels in L2.  width 0 restores the default (8); a width of at
 * least ceil(N / 128) gives the plain column-major triangle.  FP32 handles
 * accept and ignore it.  PLV_ERR_INVALID for a NULL handle or width < 0. */
plv_status plv_set_gram_raster(plv_handle *h, int width);

/* Failure detection (no counterpart in the paper).  Every wait of the
 * tensor-core Gram's pipeline (a stage of operands landing, an accumulator
 * chunk being drained) is bounded: after `ns` nanoseconds of %globaltimer
 * the CTA records PLV_ERR_TIMEOUT in the handle's device status word (read
 * by plv_sync_status), stops issuing, lets the copies and MMAs it issued
 * finish (each within its own fixed 0.1 s bound), frees its tensor memory
 * and returns; outputs of that launch are then incomplete.  The bound
 * applies to later plv_gram, plv_gram_windows, plv_gram_grouped and split-
 * precision plv_backward calls on this handle.  ns = 0 restores the default
 * of 4 s; a short bound (microseconds) exists for tests of this path.
 * PLV_ERR_INVALID for a NULL handle. */
plv_status plv_set_wait_limit(plv_handle *h, uint64_t ns);

/* Device memory the handle holds (twiddle tables, any-length and band
 * plans, backward scratch including scratch kept for captured graphs): the
 * bytes now and the most held so far, the high-water mark of the library's
 * own allocations (caller-owned tensors are not included).  NULL outputs are
 * skipped.  PLV_ERR_INVALID for a NULL handle. */
plv_status plv_memory_usage(const plv_handle *h, size_t *current, size_t *peak);

/* Bounds-checked builds (no counterpart in the paper).  The library built
 * with PLV_CHECKED (libplv_checked.so) tests the bounds conditions of the
 * index computations of the analytic-signal kernels (shared-memory
 * positions, sample ranges of the stores) and of the tensor-core Gram
 * (operand blocks copied, output rows and columns written): an access that
 * fails its condition is skipped and the source line of the first failure
 * is recorded on the device, never trapped.  plv_check_status synchronises
 * `stream`, reads the first recorded line of the handle's device into
 * *line (0: none) and clears it.  On the unchecked build it sets *line = 0.
 * PLV_ERR_INVALID for a NULL argument. */
plv_status plv_check_status(plv_handle *h, void *stream, int *line);
/* 1 for the bounds-checked build, 0 otherwise. */
int plv_build_checked(void);

/* Host-side fault injection for tests of the error paths (no counterpart in
 * the paper).  Process-wide; one fault is armed at a time, and it disarms
 * itself when it fires.  Nothing here makes a GPU fault, trap or hang.
 *   PLV_FAULT_ALLOC  the countdown-th next device allocation made by the
 *                    library (handle tables, plans, scratch, group plans)
 *                    fails as if cudaMalloc had: the call returns
 *                    PLV_ERR_ALLOC and frees what it had allocated;
 *   PLV_FAULT_LAUNCH the countdown-th next kernel launch made by an entry
 *                    point is not made and is reported as a failed launch
 *                    (PLV_ERR_CUDA);
 *   PLV_FAULT_STALL  the next tensor-core Gram launch withholds the first
 *                    operand copy of every CTA, so each CTA's bounded
 *                    pipeline wait (plv_set_wait_limit) runs out: the call
 *                    itself returns PLV_OK and the launch ends with
 *                    PLV_ERR_TIMEOUT in the device status word;
 *   PLV_FAULT_NONE   disarms.
 * countdown >= 1 (1: the next event).  The environment variable PLV_FAULT,
 * read when the library is loaded, arms the same faults: "alloc[:n]",
 * "launch[:n]" or "timeout" (the stall).  PLV_ERR_INVALID for an unknown
 * kind or countdown < 1. */
enum {
    PLV_FAULT_NONE = 0,
    PLV_FAULT_ALLOC = 1,
    PLV_FAULT_LAUNCH = 2,
    PLV_FAULT_STALL = 3
};
plv_status plv_debug_fault(int kind, int countdown);
/* The armed fault: its kind (PLV_FAULT_NONE when disarmed) and, if
 * countdown is not NULL, the events left until it fires. */
int plv_debug_fault_armed(int *countdown);

/* Row length (in elements) of the phasor operand layout for T samples: T
 * rounded up to a multiple of 32; the padding samples are zero. */
int64_t plv_phasor_ld(int T);

/* Bytes of the phasor operand buffer P for `batch` epochs of N x T (8 bytes
 * per padded sample), ld = plv_phasor_ld(T):
 *   FP32:   float P[batch][N][2][ld]: plane 0 = Re P, plane 1 = Im P.
 *   BF16X3 / FP16X3: 16-bit hi / lo splits in blocks of 128 rows x 32
 *   samples x 4 planes (Re_hi, Re_lo, Im_hi, Im_lo), 32 KB each, stored
 *   in the order [batch][ceil(N/128)][ld/32]; inside a block [plane][row]
 *   [32 samples], the four 16-byte chunks of each 64-byte row rotated by
 *   XOR with ((row >> 1) & 3) (the tensor cores' 64-byte swizzle).  Rows
 *   are padded with zeros to a multiple of 128.
 * Returns 0 for invalid sizes. */
size_t plv_phasor_bytes(const plv_handle *h, int batch, int N, int T);

/* Make the handle's per-length tables for T samples: for lengths outside the
 * direct FFT, the any-length transform's twiddles and Hilbert-kernel
 * spectrum (allocates).  The first plv_analytic call for a new T does this
 * implicitly; call it beforehand when that call is to be captured in a CUDA
 * graph. */
plv_status plv_prepare(plv_handle *h, int T);

/* Eq. 3 + Eq. 4, fused (Section II.A): analytic signal of every row of x by
 * FFT (forward transform, multiply by the analytic mask, inverse transform)
 * and unit phasors P = z/|z| written in the handle's operand layout.
 *   x    : real, [batch][N][ldx] (ldx >= T), dtype F32 or F64 (F64 is
 *          converted to FP32 on load; the arithmetic is FP32).
 *   P    : plv_phasor_bytes(h, batch, N, T) bytes, written completely
 *          (including zero padding).
 * Supported T: 2 <= T <= 12288.  Powers of two from 32 to 8192 take the
 * direct radix-16 FFT of length T; every other length takes the circular
 * convolution with the periodic Hilbert kernel through an FFT of length
 * M >= 2T - 1 (M = 2^a, 3 * 2^a or 5 * 2^a), whose tables are made on first use of a
 * T (allocates; see plv_prepare).  Others: PLV_ERR_UNSUPPORTED.
 * batch = 0 or N = 0 is a no-op. */
plv_status plv_analytic(plv_handle *h, void *stream, const void *x,
                        plv_dtype dtype, int batch, int N, int T, int64_t ldx,
                        void *P);

/* The band-pass and Eq. 3 in one transform, for several bands (the
 * band-pass then analytic signal of Section III.A), fused with Eq. 4: for
 * band b, z_b = IFFT(h B_b FFT(x)) with a real band mask B_b, then
 * P_b = z_b / |z_b| in the handle's operand layout.
 *   x     : real [batch][N][ldx] (ldx >= T), F32 or F64, broadband.
 *   masks : float [nbands][T/2 + 1] on the device: B_b at the bins
 *           0 .. T/2 (the mask of bin -k is that of k; h zeroes the negative
 *           frequencies).
 *   P     : nbands operand buffers back to back, each
 *           plv_phasor_bytes(h, batch, N, T) bytes (written completely).
 * T from 2 to 12288:
 *   - powers of two from 128 to 8192: one forward FFT per pair of rows
 *     serves every band; asynchronous, can be captured in a CUDA graph;
 *   - every other T: the circular convolution of each row with the band's
 *     kernel IDFT_T(h B_b) through one zero-padded transform of length
 *     M >= 2T - 1, one row per transform (the kernel is complex), the
 *     forward spectrum kept in the handle's scratch for all bands.  The
 *     kernels' spectra are computed on the host in FP64 from the mask
 *     values, which are read back: the call synchronises the stream,
 *     allocates on first use of a (T, masks) pair (cached by the mask
 *     values) and fails with PLV_ERR_INVALID inside a stream capture.  A
 *     sample with |z_b|^2 below 2^-40 of the row's mean x^2 counts as
 *     |z_b| = 0.
 * Others: PLV_ERR_UNSUPPORTED. */
plv_status plv_analytic_bands(plv_handle *h, void *stream, const void *x,
                              plv_dtype dtype, int batch, int N, int T, int64_t ldx,
                              const float *masks, int nbands, void *P);

/* Eq. 4 alone, for callers that already hold an analytic signal (for
 * example from a wavelet transform): P = z/|z| in the operand layout.
 *   z    : complex interleaved (re, im), [batch][N][ldz] complex elements,
 *          ldz >= T; dtype F32 (complex64) or F64 (complex128).
 * Any T >= 1. */
plv_status plv_normalize(plv_handle *h, void *stream, const void *z,
                         plv_dtype dtype, int batch, int N, int T, int64_t ldz,
                         void *P);

/* Eq. 7, 13, 14 (Section II.A, II.C): the Hermitian Gram C = P P^H / T of
 * every epoch (upper-triangle tiles only) with the read-outs fused into its
 * epilogue.
 *   P        : operand buffer written by plv_analytic / plv_normalize for the
 *              same (batch, N, T) and the same handle precision.
 *   out_mask : OR of PLV_OUT_*; an output whose bit is clear, or whose
 *              pointer is NULL, is not written.
 *   plv, iplv, ciplv : float [batch][N][N] row-major.
 *   C        : complex64 interleaved [batch][N][N] (8 bytes per entry).
 *   diag_dev : double [batch] or NULL: max_i |C_ii - 1| per epoch, the unit-
 *              modulus check of Eq. 4 (1/T applied in FP64).
 * FP64 is used only for the diagonal check.  The ciPLV denominator
 * (1 - Re C)(1 + Re C) is formed with an error-free transformation in FP32
 * (exact product via FMA, exact 1 + |Re C| via Fast2Sum): within one ulp of
 * its correctly rounded exact value, as an FP64 evaluation would give, with
 * no cancellation as |Re C| -> 1. */
plv_status plv_gram(plv_handle *h, void *stream, const void *P, int batch,
                    int N, int T, unsigned out_mask, float *plv, float *iplv,
                    float *ciplv, void *C, double *diag_dev);

/* Sliding-window Grams (dynamic PLV, Eq. 7 restricted to windows of the
 * samples): for every epoch b and window w < nw of W samples starting at
 * t0 + w * hop, C = (1/W) sum over the window of P_i conj(P_j), with the
 * read-outs of plv_gram.
 *   P        : as for plv_gram(h, stream, P, batch, N, T, ...).
 *   t0, W, hop: multiples of 32 (the operand layout's sample blocks), W >= 32,
 *              and every window inside the T samples:
 *              t0 + (nw - 1) * hop + W <= T.
 *   outputs  : [batch][nw][N][N] (diag_dev: [batch][nw]); layouts and NULL
 *              handling as in plv_gram.
 * Errors: PLV_ERR_INVALID. */
plv_status plv_gram_windows(plv_handle *h, void *stream, const void *P, int batch, int N,
                            int T, int t0, int W, int hop, int nw, unsigned out_mask,
                            float *plv, float *iplv, float *ciplv, void *C, double *diag_dev);

/* One problem of a grouped plan: its phasors P for (batch, N, T) in the
 * handle's operand layout, its Gram outputs (layouts as in plv_gram; NULL
 * outputs are skipped) and, optionally, its real input x for
 * plv_analytic_grouped.  With x NULL the phasors are written by the caller
 * (plv_analytic / plv_normalize of the same handle). */
typedef struct {
    void *P;
    int batch, N, T;
    float *plv, *iplv, *ciplv;
    void *C;          /* complex64 [batch][N][N] */
    double *diag;     /* [batch] */
    const void *x;    /* real [batch][N][ldx] or NULL */
    int64_t ldx;      /* row stride of x in elements, >= T */
    plv_dtype dtype;  /* PLV_F32 or PLV_F64; one dtype for every x of a plan */
} plv_problem;

typedef struct plv_group plv_group;

/* Plan a grouped run over `nprob` problems of uneven N and T (Section IV:
 * many subjects, epochs and frequency bands): uploads the problem
 * descriptors and the list of every (problem, epoch, upper-triangle tile),
 * sorted longest first (by T), to the device; for the problems with an
 * input x also the list of every (problem, row pair) of the analytic-signal
 * engine, and, for the split precisions, zeroes the padding rows of their P
 * once (no call writes them later).  Allocates and synchronises the device:
 * call outside stream capture.  out_mask selects outputs as in plv_gram.
 * The pointers in `probs` are captured: the plan runs on those buffers.  The
 * plan uses tables owned by the handle and must not outlive it. */
plv_status plv_group_create(plv_handle *h, const plv_problem *probs, int nprob,
                            unsigned out_mask, plv_group **group);

/* Run a plan: Eq. 7, 13, 14 for every problem.  BF16X3 / FP16X3 handles run
 * ONE persistent tensor-core launch over the whole tile list (CTAs take
 * tiles round-robin, longest first), preceded by a memset of the split-K
 * counters when the plan splits tiles; an FP32 handle runs one Gram launch
 * per problem.  Allocates nothing: can be captured in a CUDA graph.  Two
 * runs of one plan must not overlap (on two streams): they write the same
 * outputs and share the split counters. */
plv_status plv_gram_grouped(plv_handle *h, void *stream, const plv_group *group);

/* Eq. 3 and 4 for every problem of a plan that has an input x: the
 * analytic signal by the any-length engine of plv_analytic (also for
 * power-of-two T, whose results may then differ from plv_analytic's in the
 * last bits) fused with the unit-phasor normalisation, written to the
 * problem's P.  One persistent launch per thread class of the engine (at most
 * four), each over all (problem, row pair) of the class, longest transform
 * first.  Allocates nothing: can be captured in a CUDA graph.  Fails with
 * PLV_ERR_INVALID if the plan has no input. */
plv_status plv_analytic_grouped(plv_handle *h, void *stream, const plv_group *group);

/* What plv_group_tune chose and measured.  Times are medians of `reps`
 * launches in milliseconds (0 where nothing was timed); "default" is the
 * plan's configuration when the call began. */
typedef struct {
    float k1_ms_default, k1_ms_tuned;      /* plv_analytic_grouped's launches */
    float gram_ms_default, gram_ms_tuned;  /* plv_gram_grouped's launch (split precisions) */
    int k1_lengths;     /* distinct transform lengths M of the plan's analytic signal */
    int k1_widened;     /* lengths moved to the next wider thread class (2x threads per transform) */
    int k1_per_sm[4];   /* CTAs per SM of each thread class launch; 0: the occupancy limit */
    int k1_launches;    /* non-empty thread class launches of plv_analytic_grouped */
    int gram_schedule;  /* 0: longest first, round-robin; 1: balanced rounds */
    int gram_tile_cost; /* per-tile cost (in 32-sample K blocks) the balanced rounds assumed */
    int gram_split;     /* split-K factor f kept (0: no tile split; plv_group_configure) */
    int gram_split_tiles; /* tiles that run as several parts under it */
    int timed_configs;  /* configurations launched and timed */
    int cached;         /* 1: the configuration came from the handle's cache; nothing was timed */
} plv_tune_result;

/* Autotuner of a grouped plan (the batching of Section IV's many subjects
 * and bands; the paper has no GPU design to follow here).  Times, with CUDA
 * events on `stream`, candidate launch shapes that leave every result the
 * same and keeps the fastest in the plan:
 *   - analytic signal: for each transform length M, the CTA width of the
 *     any-length engine (its own thread class or the next wider one, timed
 *     on that length's rows alone), then the CTAs per SM of each class
 *     launch; the tuned set is kept only if the whole grouped launch is
 *     faster than the default;
 *   - Gram (BF16X3 / FP16X3): the tile schedule, i.e. the order of the
 *     tile list that the persistent CTAs take round-robin: longest first
 *     (default) or balanced rounds (each round of G tiles dealt to the
 *     least-loaded CTAs under a per-tile cost of 0, 8 or 32 K blocks); then,
 *     in that schedule, split K with factor f = 1, 2 or 4 (see
 *     plv_gram_split_plan and plv_group_configure), kept if 3 % faster.
 * The candidates run on the plan's own buffers and write the plan's outputs
 * (with the values any run writes), so the phasors P must be valid for the
 * Gram part: with an input x the tuner's own analytic-signal launches write
 * them, without one the caller must have.  reps (1..100) timed launches per
 * candidate.  The choice is cached in the handle under the plan's work
 * signature (precision, SM count, transform lengths, tile K lengths): tuning
 * an equal plan applies it without timing (result->cached = 1).
 * Synchronises the device and allocates the new work lists: call outside
 * stream capture (PLV_ERR_INVALID otherwise) and while no launch of the plan
 * is in flight.  CUDA graphs captured before tuning keep their old lists
 * (kept alive until plv_group_destroy) and so the old configuration.
 * result may be NULL. */
plv_status plv_group_tune(plv_handle *h, void *stream, plv_group *group, int reps,
                          plv_tune_result *result);

/* Set a plan's launch shapes without timing (to pin or reproduce one of
 * the tuner's candidates; the paper has no counterpart):
 *   k1_widen       0: every transform length in its own thread class;
 *                  1: every length in the next wider class (the widest
 *                     class stays);
 *   k1_per_sm      [4] CTAs per SM of each class launch (0: the occupancy
 *                  limit; values above it act as 0), or NULL for all 0;
 *   gram_schedule  0: longest first; 1: balanced rounds with per-tile cost
 *                  gram_tile_cost (0 .. 2^20 K blocks);
 *   gram_split     split-K factor f (0 .. 64; 0: no tile split): tiles longer
 *                  than the grid's fair share / f (and than 2048 samples) run
 *                  as several parts on different CTAs (plv_gram_split_plan).
 *                  A part sums its K range as a whole tile does and stores
 *                  the sums in a 128 KB slot of the plan; for each 32 x 32
 *                  block, the last part to finish adds the tile's slots in
 *                  part order and stores the block.  The plan allocates the
 *                  slots (at most 8192, 1 GiB) and 16 counters per split
 *                  tile.
 * Results do not depend on the K1 shapes and the schedule: they give the
 * same bits.  Split K regroups a split tile's FP32 additions (part sums,
 * then their sum in part order), so its results differ from the unsplit
 * plan's by FP32 rounding; a given configuration gives the same bits on
 * every run.  Same synchronisation, allocation and graph rules as
 * plv_group_tune.  Errors: PLV_ERR_INVALID for values out of range. */
plv_status plv_group_configure(plv_handle *h, void *stream, plv_group *group, int k1_widen,
                               const int *k1_per_sm, int gram_schedule, int gram_tile_cost,
                               int gram_split);

/* The split-K plan of plv_group_configure and plv_group_tune (host only;
 * needs no device).  For ntiles tiles of nkb[i] 32-sample K blocks, `chunk`
 * K blocks per summation chunk (32 for BF16X3, 4 for FP16X3), a persistent
 * grid of `grid` CTAs and factor `split` (0 .. 64), writes parts[i], the
 * number of parts tile i runs as (1: whole).  With W the total K blocks and
 * L = max(chunk, 64, ceil(W / (grid split))), a tile of nkb > L K blocks
 * takes S = min(ceil(nkb / L), ceil(nkb / chunk)) parts, longest tiles
 * first while the slots (8192, one per part) last; part s of S covers the
 * chunks [floor(s nch / S), floor((s + 1) nch / S)) of the tile's nch.
 * split = 0 gives 1 everywhere.  Errors: PLV_ERR_INVALID. */
plv_status plv_gram_split_plan(const int *nkb, int ntiles, int chunk, int grid, int split,
                               int *parts);

/* Free a plan (synchronises the device).  NULL is ignored. */
plv_status plv_group_destroy(plv_group *group);

/* Eq. 7, 13, 14 applied elementwise to a stored C (complex64 interleaved,
 * [batch][N][N]); the same arithmetic as the fused epilogue, including the
 * zero diagonal of iPLV / ciPLV.  NULL outputs are skipped. */
plv_status plv_metrics(plv_handle *h, void *stream, const void *C, int batch,
                       int N, float *plv, float *iplv, float *ciplv);

/* Gradient of L = sum_ij (g_plv PLV + g_iplv iPLV + g_ciplv ciPLV)_ij with
 * respect to the real input x, through Eq. 14, 13, 7 (read-outs and Gram),
 * Eq. 4 (normalisation) and Eq. 3 (analytic signal).  The analytic signal is
 * recomputed from x (it is not stored by the forward pass).
 *   x        : the forward input, [batch][N][ldx], F32 or F64.
 *   C        : complex64 [batch][N][N], the forward Gram (plv_gram with
 *              PLV_OUT_C, any precision).
 *   g_plv, g_iplv, g_ciplv : float [batch][N][N] upstream gradients of the
 *              three outputs; NULL means zero.  Diagonal entries are ignored
 *              (the forward diagonal does not depend on x).
 *   grad_x   : float [batch][N][T] (row stride T), written completely.
 * Conventions: dPLV/dC = C/|C| (0 at |C| = 0); d|Im C|/dIm C = sign(Im C)
 * (0 at 0); ciPLV is differentiated where (1 - Re C)(1 + Re C) > 0.
 * Arithmetic FP32, except the one dense contraction Gamma = S P / T
 * (S = G + G^H): on an FP32 handle FP32 FMA on the CUDA cores; on a BF16X3
 * or FP16X3 handle the tensor cores, with S and P as BF16 hi + lo splits
 * and three products per term (BF16 for both handle kinds: gradients can
 * exceed the FP16 range).  Supported T: as plv_analytic.  Uses handle
 * scratch of batch*N*ld*20 bytes plus, on an FP32 handle, batch*N*N*8, or,
 * on a split handle, batch*ceil(N/128)*128*(32*ceil(N/32) + ld)*8;
 * allocated on first use for a size (cudaMalloc; fails with PLV_ERR_INVALID
 * if that first use is inside a stream capture).  A CUDA graph captured
 * with this call keeps using the scratch it was captured with: when a later,
 * larger call (outside capture) grows the scratch, a buffer that a capture
 * used is kept, still counted against the workspace limit, until
 * plv_destroy, so replaying the older graph stays valid. */
plv_status plv_backward(plv_handle *h, void *stream, const void *x,
                        plv_dtype dtype, int batch, int N, int T, int64_t ldx,
                        const void *C, const float *g_plv, const float *g_iplv,
                        const float *g_ciplv, float *grad_x);

/* The forward pass in the form that lets the backward pass skip its
 * recompute (no counterpart in the paper; the trade of memory for time that
 * plv_backward makes the other way): Eq. 3 and 4 as in plv_analytic, and
 * what the gradient of Eq. 4 needs.
 *   P    : the Gram operand for plv_gram on this handle (plv_phasor_bytes
 *          bytes; on an FP32 handle the FP32 planar phasors, on a BF16X3
 *          handle the tiled BF16 split layout, padding rows zeroed);
 *   P32  : float [batch*N][2][ld] FP32 planar phasors (on an FP32 handle
 *          P itself: pass P or NULL);
 *   rinv : float [batch*N][ld], 1/|z| (0 where |z| counts as 0, reading c7).
 * The phasors are those of plv_backward's recompute (one Newton step on
 * 1/|z|), so on a BF16X3 handle they can differ in the last bits from
 * plv_analytic's.  FP16X3 handles: PLV_ERR_UNSUPPORTED.  Supported T, x and
 * capture rules as plv_analytic. */
plv_status plv_analytic_save(plv_handle *h, void *stream, const void *x, plv_dtype dtype,
                             int batch, int N, int T, int64_t ldx, void *P, float *P32,
                             float *rinv);

/* plv_backward from what plv_analytic_save wrote (P, P32, rinv of the same
 * x), without the recompute of the analytic signal: the same gradient, bit
 * for bit, as plv_backward gives for that x and C.  Arguments, conventions,
 * arithmetic and errors as plv_backward; handle scratch of batch*N*ld*8
 * bytes plus, on an FP32 handle, batch*N*N*8, or, on a BF16X3 handle,
 * batch*ceil(N/128)*128*ceil(N/32)*32*8.  FP16X3 handles:
 * PLV_ERR_UNSUPPORTED. */
plv_status plv_backward_saved(plv_handle *h, void *stream, int batch, int N, int T,
                              const void *P, const float *P32, const float *rinv, const void *C,
                              const float *g_plv, const float *g_iplv, const float *g_ciplv,
                              float *grad_x);

/* Normalisation of plv_trial_operands. */
enum {
    PLV_TRIAL_ASIS = 0, /* values as given (unit phasors: Eq. 1 / Eq. 8)  */
    PLV_TRIAL_RMS = 1   /* divided by their RMS over trials (Eq. 12)     */
};

/* Operands of a Gram over trials, one problem per column l (a time sample
 * or a frequency bin).  The time-resolved PLV of Lachaux et al. (Eq. 1;
 * Eq. 8 is its matrix form) and coherency across trials (Eq. 12) are the
 * Gram of Eq. 7 with the E trials as the summation index:
 *   V    : float, FP32 planar rows [E][N][2][ldv] (Re plane, Im plane), the
 *          layout an FP32 handle's plv_analytic / plv_normalize writes, or
 *          any per-trial complex values in that layout (e.g. from
 *          plv_dft_bins).
 *   l0, L: the columns taken, 0 <= l0 and l0 + L <= ldv.
 *   mode : PLV_TRIAL_ASIS: row i of problem l is (V[0][i][l0+l], ...,
 *          V[E-1][i][l0+l]).  With unit phasors, plv_gram then gives the
 *          time-resolved PLV, iPLV and ciPLV of Eq. 1, 13, 14 (1/E over the
 *          trials).
 *          PLV_TRIAL_RMS: each row divided by sqrt(mean_n |V[n][i][l0+l]|^2)
 *          first (a zero row stays zero).  plv_gram then gives the coherency
 *          of Eq. 12, its magnitude (coherence), |Im| (imaginary coherency)
 *          and Im / sqrt(1 - Re^2) (lagged coherence).
 *   P    : plv_phasor_bytes(h, L, N, E) bytes in the handle's operand layout,
 *          written completely: the input of plv_gram(h, stream, P, L, N, E,
 *          ...), whose outputs are [L][N][N].
 * 1 <= E, 0 <= N <= 65408.  Errors: PLV_ERR_INVALID (sizes, NULL or
 * misaligned pointers: V 4-byte, P 16-byte), PLV_ERR_UNSUPPORTED (N). */
plv_status plv_trial_operands(plv_handle *h, void *stream, const float *V, int E, int N,
                              int64_t ldv, int l0, int L, int mode, void *P);

/* The DFT of real rows at F consecutive bins (the Fourier coefficients of
 * Eq. 10-12):  X[r][f] = sum_t x[r][t] exp(-2 pi i (f0 + f) t / T).
 *   x    : real [rows][ldx] (ldx >= T), F32 or F64 (converted to FP32).
 *   X    : float, FP32 planar rows [rows][2][ldX] (ldX >= F): Re in
 *          columns 0..F-1 of plane 0, Im in plane 1; columns F..ldX-1 are not
 *          written.  With rows = E * N this is the V of plv_trial_operands
 *          (ldv = ldX), whose mode PLV_TRIAL_RMS then gives coherency across
 *          the E trials (Eq. 12).
 * FP32 arithmetic on the CUDA cores: twiddles from the exact phase index
 * ((f0 + f) t) mod T, partial sums per 32 samples.  1 <= T <= 32768,
 * 0 <= f0, 1 <= F, f0 + F <= T.  Errors: PLV_ERR_INVALID. */
plv_status plv_dft_bins(plv_handle *h, void *stream, const void *x, plv_dtype dtype, int rows,
                        int T, int64_t ldx, int f0, int F, float *X, int64_t ldX);

/* Size of the fixed scratch array behind plv_backward_noalloc: 64 MiB. */
#define PLV_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)

/* plv_backward without any allocation and without a handle.  The paper has
 * no counterpart to this entry point; it exists for callers that cannot call
 * cudaMalloc, for example:
 *   - a plugin run inside another framework's execution engine that forbids
 *     allocation during its enqueue step;
 *   - a host whose device memory is already owned by a pooling allocator
 *     that must not be bypassed;
 *   - a latency-critical loop that must not pay for (or risk failing) an
 *     allocation.
 * Instead of handle scratch it uses one fixed device array of
 * PLV_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until
 * the process exits (plus the FFT twiddle tables, also static).
 *
 * Arguments as plv_backward (minus the handle); it runs on the CURRENT
 * device, with the arithmetic of an FP32 handle's plv_backward (FP32, the
 * contraction on the CUDA cores), whose result it equals bit for bit.  T
 * must be a power of two from 32 to 8192 (other lengths, which plv_backward
 * takes through its any-length plans, give PLV_ERR_UNSUPPORTED).  A problem
 * whose scratch (batch*N*ld*20 + batch*N*N*8
 * bytes, each of the four parts rounded up to 256 bytes; ld = plv_phasor_ld(T))
 * exceeds the array is rejected with PLV_ERR_INVALID and a message naming
 * the sizes; nothing is launched.  For example batch = 4, N = 128, T = 4096
 * fits.
 *
 * The first call on each device sets that device up: it looks up the
 * array's device address and uploads the twiddle tables (synchronous
 * copies).  Make that first call outside any stream capture.  The set-up
 * is kept for the life of the process: after a reset of a device's context
 * (cudaDeviceReset) the addresses it holds are stale, so do not call this
 * entry point on that device again.
 *
 * All calls share the one array.  Each call writes every scratch element it
 * reads, so no clearing is needed between calls.  Calls whose work overlaps
 * on the GPU (different streams, or graphs replayed concurrently) race on
 * the array and corrupt each other's results: serialise them.
 * plv_last_error(NULL) returns the message of a failure. */
plv_status plv_backward_noalloc(void *stream, const void *x, plv_dtype dtype,
                                int batch, int N, int T, int64_t ldx,
                                const void *C, const float *g_plv,
                                const float *g_iplv, const float *g_ciplv,
                                float *grad_x);

/* Read (and clear) the handle's device status word after synchronising
 * `stream`.  *device_status receives PLV_OK or the recorded error. */
plv_status plv_sync_status(plv_handle *h, void *stream, int *device_status);

#ifdef __cplusplus
}
#endif

#endif /* PLV_H */
