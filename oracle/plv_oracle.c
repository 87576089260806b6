/*
 * plv_oracle.c -- plain FP64 CPU oracle for the reformulated Phase Locking
 * Value (Bruna, Maestu & Pereda, "Phase Locking Value revisited").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or helper
 * with the CUDA path.
 *
 * What it computes, step by step, in the paper's order:
 *   1. the analytic signal of every row by a direct O(T^2) DFT (Section II.A,
 *      Eq. 3): X[k] = sum_t x[t] w^{kt}, w = exp(-2 pi i / T); Z = h (.) X;
 *      z[t] = (1/T) sum_k Z[k] w^{-kt}.  h is the standard discrete analytic
 *      signal mask (the paper names the Hilbert analytic signal but not the
 *      discrete mask): even T: h[0]=h[T/2]=1, h[1..T/2-1]=2, 0 elsewhere;
 *      odd T: h[0]=1, h[1..(T-1)/2]=2, 0 elsewhere.
 *   2. the instantaneous phase phi = atan2(Im z, Re z) (the phase extraction
 *      that the paper's original implementation performs, Appendix).
 *   3. the original pairwise definition (Eq. 2, time-averaged PLV / mean
 *      phase coherence): c_ij = (1/T) sum_t exp(i (phi_i(t) - phi_j(t))),
 *      evaluated for every ordered pair (i, j), diagonal included.
 *   4. the read-outs: PLV = |c| (Eq. 2 / Eq. 7), iPLV = |Im c| (Eq. 13, taken
 *      in absolute value), ciPLV = Im c / sqrt((1 - Re c)(1 + Re c)) (Eq. 14).
 *   5. separately, for the equivalence check only, the reformulated
 *      definition (Eq. 5-7): c_ij = (1/T) sum_t z_i conj(z_j) / (|z_i||z_j|).
 *
 * Readings where the paper is silent:
 *   - a sample with |z| = 0 has no phase; its unit phasor is taken as 0, so
 *     the sample contributes nothing to any pair (Eq. 4 divides by |z|).
 *   - where (1 - Re c)(1 + Re c) <= 0 (the diagonal, exact zero-lag copies),
 *     ciPLV is defined as 0 (Eq. 14 is undefined there).
 *   - the diagonal of iPLV and ciPLV is 0 by definition (Im c_ii = 0).
 *
 * Extensions over trials (the time-resolved PLV and coherency across trials):
 *   6. the time-resolved PLV of Lachaux et al. (Eq. 1; Eq. 8 is its matrix
 *      form): for every sample t, c_ij(t) = (1/E) sum_n exp(i (phi_i(t, n) -
 *      phi_j(t, n))) over the E trials n, then the read-outs of step 4;
 *   7. the DFT of real rows at selected bins, X[f] = sum_t x[t] w^{f t}
 *      (the Fourier coefficients of Eq. 10-12), by the direct sum;
 *   9. the analytic signal of a band-passed row, band-pass and analytic
 *      mask in one transform: z = IDFT(h B DFT(x)) for a real band mask B
 *      (the band-pass then analytic signal of Section III.A);
 *   8. coherency across trials (Eq. 12): coh_ij = sum_n X_i(n) conj(X_j(n)) /
 *      sqrt(sum_n |X_i(n)|^2 sum_n |X_j(n)|^2), with the read-outs of step 4
 *      (coherence |coh|, imaginary coherency |Im coh|, lagged coherence
 *      Im coh / sqrt(1 - (Re coh)^2)); a channel of zero power has coh = 0.
 *
 * Parity is pinned (tests/test_oracle.py) against scipy's FFT-based analytic
 * signal, closed forms for on-bin tones and lagged tones, brute force, and
 * statistical invariants.  No function here is "parity unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Number of OpenMP threads the oracle may use (0 = library default). */
static int g_threads = 0;

void oracle_set_threads(int n) { g_threads = n; }

int oracle_max_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* Analytic-signal mask h[k] of step 1 (Eq. 3 via the discrete analytic
 * signal).  Returns 0, 1 or 2. */
static double hmask(long k, long T) {
    if (k == 0) return 1.0;
    if (T % 2 == 0) {
        if (k == T / 2) return 1.0;
        return (k < T / 2) ? 2.0 : 0.0;
    }
    return (k <= (T - 1) / 2) ? 2.0 : 0.0;
}

/*
 * Step 1 (Eq. 3): analytic signal of `rows` real rows of length T.
 * x: rows x T (row stride ldx).  z_re, z_im: rows x T (row stride T).
 * Direct DFT; twiddles from an FP64 table tw[m] = exp(-2 pi i m / T), indexed
 * by (k t) mod T so the argument never grows.  Returns 0, or -1 on bad args.
 */
static int analytic_impl(const double *x, long rows, long T, long ldx,
                         const double *band, double *z_re, double *z_im) {
    if (rows < 0 || T < 1 || ldx < T) return -1;
    if (rows == 0) return 0;
    double *twc = (double *)malloc(sizeof(double) * (size_t)T);
    double *tws = (double *)malloc(sizeof(double) * (size_t)T);
    if (!twc || !tws) { free(twc); free(tws); return -1; }
    for (long m = 0; m < T; ++m) {
        double a = 2.0 * M_PI * (double)m / (double)T;
        twc[m] = cos(a);
        tws[m] = -sin(a); /* w^m = cos - i sin */
    }
    long K = T / 2 + 1; /* h[k] = 0 beyond k = floor(T/2) */
    int nt = oracle_max_threads();
    int fail = 0;
#pragma omp parallel num_threads(nt)
    {
        double *Xr = (double *)malloc(sizeof(double) * (size_t)K);
        double *Xi = (double *)malloc(sizeof(double) * (size_t)K);
        if (!Xr || !Xi) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (long r = 0; r < rows; ++r) {
                const double *xr = x + r * ldx;
                /* forward DFT, only the bins h keeps */
                for (long k = 0; k < K; ++k) {
                    double sr = 0.0, si = 0.0;
                    long idx = 0; /* (k t) mod T */
                    for (long t = 0; t < T; ++t) {
                        sr += xr[t] * twc[idx];
                        si += xr[t] * tws[idx];
                        idx += k;
                        if (idx >= T) idx -= T;
                    }
                    double h = hmask(k, T) * (band ? band[k] : 1.0);
                    Xr[k] = h * sr;
                    Xi[k] = h * si;
                }
                /* inverse DFT: z[t] = (1/T) sum_k Z[k] w^{-kt} */
                for (long t = 0; t < T; ++t) {
                    double sr = 0.0, si = 0.0;
                    long idx = 0; /* (k t) mod T */
                    for (long k = 0; k < K; ++k) {
                        /* w^{-m} = cos + i sin = twc - i tws */
                        double c = twc[idx], s = -tws[idx];
                        sr += Xr[k] * c - Xi[k] * s;
                        si += Xr[k] * s + Xi[k] * c;
                        idx += t;
                        if (idx >= T) idx -= T;
                    }
                    z_re[r * T + t] = sr / (double)T;
                    z_im[r * T + t] = si / (double)T;
                }
            }
        }
        free(Xr);
        free(Xi);
    }
    free(twc);
    free(tws);
    return fail ? -1 : 0;
}

int oracle_analytic(const double *x, long rows, long T, long ldx,
                    double *z_re, double *z_im) {
    return analytic_impl(x, rows, T, ldx, NULL, z_re, z_im);
}

/*
 * Step 9: the analytic signal of the band-passed rows, the band-pass and the
 * analytic mask applied in one transform: Z[k] = h[k] B[k] X[k] with a real
 * band mask B on the bins k = 0 .. floor(T/2) (B[k] for the negative
 * frequency -k is irrelevant, h being 0 there), then the inverse DFT as in
 * step 1.  band: floor(T/2) + 1 values.
 */
int oracle_analytic_band(const double *x, long rows, long T, long ldx,
                         const double *band, double *z_re, double *z_im) {
    if (!band) return -1;
    return analytic_impl(x, rows, T, ldx, band, z_re, z_im);
}

/* Step 4 (Eq. 7, 13, 14): read-outs of one complex c. */
static void readout(double cr, double ci, double *plv, double *iplv,
                    double *ciplv) {
    *plv = sqrt(cr * cr + ci * ci);
    *iplv = fabs(ci);
    double d = (1.0 - cr) * (1.0 + cr);
    *ciplv = (d > 0.0) ? ci / sqrt(d) : 0.0;
}

/*
 * Steps 2-4 for selected rows: the original pairwise definition (Eq. 2) for
 * pairs (rows[r], j), j = 0..N-1.  z: N x T complex (planar re / im, row
 * stride T).  Outputs are nrows x N (row stride N); any output pointer may be
 * NULL.  c_re / c_im receive the complex mean c itself.
 */
int oracle_plv_pairwise_rows(const double *z_re, const double *z_im, long N,
                             long T, const long *rows, long nrows,
                             double *c_re, double *c_im, double *plv,
                             double *iplv, double *ciplv) {
    if (N < 0 || T < 1 || nrows < 0) return -1;
    for (long r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= N) return -1;
    if (N == 0 || nrows == 0) return 0;
    /* step 2: phases, and which samples have a phase at all */
    double *phi = (double *)malloc(sizeof(double) * (size_t)(N * T));
    unsigned char *has = (unsigned char *)malloc((size_t)(N * T));
    if (!phi || !has) { free(phi); free(has); return -1; }
    int nt = oracle_max_threads();
#pragma omp parallel for num_threads(nt) schedule(static)
    for (long q = 0; q < N * T; ++q) {
        double a = z_re[q], b = z_im[q];
        has[q] = (a != 0.0 || b != 0.0);
        phi[q] = atan2(b, a);
    }
    /* step 3: c_ij = (1/T) sum_t exp(i (phi_i - phi_j)) */
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1) collapse(2)
    for (long r = 0; r < nrows; ++r) {
        for (long j = 0; j < N; ++j) {
            long i = rows[r];
            const double *pi = phi + i * T, *pj = phi + j * T;
            const unsigned char *hi = has + i * T, *hj = has + j * T;
            double sr = 0.0, si = 0.0;
            for (long t = 0; t < T; ++t) {
                if (!(hi[t] && hj[t])) continue; /* |z| = 0: no phase */
                double d = pi[t] - pj[t];
                sr += cos(d);
                si += sin(d);
            }
            double cr = sr / (double)T, ci = si / (double)T;
            long o = r * N + j;
            if (c_re) c_re[o] = cr;
            if (c_im) c_im[o] = ci;
            double p, ip, cp;
            readout(cr, ci, &p, &ip, &cp);
            if (i == j) { ip = 0.0; cp = 0.0; } /* Im c_ii = 0 exactly */
            if (plv) plv[o] = p;
            if (iplv) iplv[o] = ip;
            if (ciplv) ciplv[o] = cp;
        }
    }
    free(phi);
    free(has);
    return 0;
}

/* Steps 2-4 for all N x N ordered pairs. */
int oracle_plv_pairwise(const double *z_re, const double *z_im, long N, long T,
                        double *c_re, double *c_im, double *plv, double *iplv,
                        double *ciplv) {
    if (N < 0) return -1;
    if (N == 0) return 0;
    long *rows = (long *)malloc(sizeof(long) * (size_t)N);
    if (!rows) return -1;
    for (long i = 0; i < N; ++i) rows[i] = i;
    int rc = oracle_plv_pairwise_rows(z_re, z_im, N, T, rows, N, c_re, c_im,
                                      plv, iplv, ciplv);
    free(rows);
    return rc;
}

/*
 * Step 5 (Eq. 5-7), the reformulation, written as a plain loop for the
 * equivalence check: c_ij = (1/T) sum_t z_i(t) conj(z_j(t)) / (|z_i||z_j|),
 * a sample with |z| = 0 contributing 0.  Outputs N x N complex (planar).
 */
int oracle_gram_direct(const double *z_re, const double *z_im, long N, long T,
                       double *c_re, double *c_im) {
    if (N < 0 || T < 1) return -1;
    int nt = oracle_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1) collapse(2)
    for (long i = 0; i < N; ++i) {
        for (long j = 0; j < N; ++j) {
            double sr = 0.0, si = 0.0;
            for (long t = 0; t < T; ++t) {
                double ar = z_re[i * T + t], ai = z_im[i * T + t];
                double br = z_re[j * T + t], bi = z_im[j * T + t];
                double na = sqrt(ar * ar + ai * ai), nb = sqrt(br * br + bi * bi);
                if (na == 0.0 || nb == 0.0) continue;
                /* (ar + i ai)(br - i bi) */
                sr += (ar * br + ai * bi) / (na * nb);
                si += (ai * br - ar * bi) / (na * nb);
            }
            c_re[i * N + j] = sr / (double)T;
            c_im[i * N + j] = si / (double)T;
        }
    }
    return 0;
}

/* Step 4 alone, elementwise over n complex values (Eq. 7, 13, 14). */
int oracle_metrics(const double *c_re, const double *c_im, long n, double *plv,
                   double *iplv, double *ciplv) {
    if (n < 0) return -1;
    for (long q = 0; q < n; ++q) {
        double p, ip, cp;
        readout(c_re[q], c_im[q], &p, &ip, &cp);
        if (plv) plv[q] = p;
        if (iplv) iplv[q] = ip;
        if (ciplv) ciplv[q] = cp;
    }
    return 0;
}

/*
 * Step 6: the time-resolved PLV (Eq. 1 / Eq. 8) for samples t0 .. t0+L-1.
 * z: E x N x T complex (planar re / im, row stride T).  Outputs L x N x N
 * (row stride N, matrix stride N*N); any output pointer may be NULL.  A
 * sample with |z| = 0 has no phase and contributes nothing (the normaliser
 * stays 1/E).
 */
int oracle_plv_time_resolved(const double *z_re, const double *z_im, long E,
                             long N, long T, long t0, long L, double *c_re,
                             double *c_im, double *plv, double *iplv,
                             double *ciplv) {
    if (E < 1 || N < 0 || T < 1 || L < 0 || t0 < 0 || t0 + L > T) return -1;
    if (N == 0 || L == 0) return 0;
    int nt = oracle_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1) collapse(2)
    for (long l = 0; l < L; ++l) {
        for (long i = 0; i < N; ++i) {
            const long t = t0 + l;
            for (long j = 0; j < N; ++j) {
                double sr = 0.0, si = 0.0;
                for (long n = 0; n < E; ++n) {
                    const long qi = (n * N + i) * T + t, qj = (n * N + j) * T + t;
                    if ((z_re[qi] == 0.0 && z_im[qi] == 0.0) ||
                        (z_re[qj] == 0.0 && z_im[qj] == 0.0))
                        continue;
                    const double d = atan2(z_im[qi], z_re[qi]) - atan2(z_im[qj], z_re[qj]);
                    sr += cos(d);
                    si += sin(d);
                }
                const double cr = sr / (double)E, ci = si / (double)E;
                const long o = (l * N + i) * N + j;
                if (c_re) c_re[o] = cr;
                if (c_im) c_im[o] = ci;
                double p, ip, cp;
                readout(cr, ci, &p, &ip, &cp);
                if (i == j) { ip = 0.0; cp = 0.0; }
                if (plv) plv[o] = p;
                if (iplv) iplv[o] = ip;
                if (ciplv) ciplv[o] = cp;
            }
        }
    }
    return 0;
}

/*
 * Step 7: X[r][f] = sum_t x[r][t] exp(-2 pi i (f0 + f) t / T) for f < F, by
 * the direct sum with an FP64 twiddle table indexed ((f0 + f) t) mod T.
 * x: rows x T (row stride ldx); X planar re / im, rows x F.
 */
int oracle_dft_bins(const double *x, long rows, long T, long ldx, long f0,
                    long F, double *X_re, double *X_im) {
    if (rows < 0 || T < 1 || ldx < T || F < 0 || f0 < 0) return -1;
    double *twc = (double *)malloc(sizeof(double) * (size_t)T);
    double *tws = (double *)malloc(sizeof(double) * (size_t)T);
    if (!twc || !tws) { free(twc); free(tws); return -1; }
    for (long m = 0; m < T; ++m) {
        twc[m] = cos(2.0 * M_PI * (double)m / (double)T);
        tws[m] = -sin(2.0 * M_PI * (double)m / (double)T);
    }
    int nt = oracle_max_threads();
#pragma omp parallel for num_threads(nt) schedule(static)
    for (long r = 0; r < rows; ++r) {
        for (long f = 0; f < F; ++f) {
            const long k = (f0 + f) % T;
            double sr = 0.0, si = 0.0;
            for (long t = 0; t < T; ++t) {
                const long m = (k * t) % T;
                sr += x[r * ldx + t] * twc[m];
                si += x[r * ldx + t] * tws[m];
            }
            X_re[r * F + f] = sr;
            X_im[r * F + f] = si;
        }
    }
    free(twc);
    free(tws);
    return 0;
}

/*
 * Step 8: coherency across trials (Eq. 12) for every column l < L (a
 * frequency bin, or any per-trial complex value).  X: E x N x L complex
 * (planar, row stride L).  Outputs L x N x N as in step 6.
 */
int oracle_coherency_trials(const double *x_re, const double *x_im, long E,
                            long N, long L, double *c_re, double *c_im,
                            double *coh, double *icoh, double *lcoh) {
    if (E < 1 || N < 0 || L < 0) return -1;
    if (N == 0 || L == 0) return 0;
    int nt = oracle_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1) collapse(2)
    for (long l = 0; l < L; ++l) {
        for (long i = 0; i < N; ++i) {
            double pii = 0.0;
            for (long n = 0; n < E; ++n) {
                const long q = (n * N + i) * L + l;
                pii += x_re[q] * x_re[q] + x_im[q] * x_im[q];
            }
            for (long j = 0; j < N; ++j) {
                double sr = 0.0, si = 0.0, pjj = 0.0;
                for (long n = 0; n < E; ++n) {
                    const long qi = (n * N + i) * L + l, qj = (n * N + j) * L + l;
                    /* X_i conj(X_j) */
                    sr += x_re[qi] * x_re[qj] + x_im[qi] * x_im[qj];
                    si += x_im[qi] * x_re[qj] - x_re[qi] * x_im[qj];
                    pjj += x_re[qj] * x_re[qj] + x_im[qj] * x_im[qj];
                }
                const double den = sqrt(pii * pjj);
                const double cr = den > 0.0 ? sr / den : 0.0;
                const double ci = den > 0.0 ? si / den : 0.0;
                const long o = (l * N + i) * N + j;
                if (c_re) c_re[o] = cr;
                if (c_im) c_im[o] = ci;
                double p, ip, cp;
                readout(cr, ci, &p, &ip, &cp);
                if (i == j) { ip = 0.0; cp = 0.0; }
                if (coh) coh[o] = p;
                if (icoh) icoh[o] = ip;
                if (lcoh) lcoh[o] = cp;
            }
        }
    }
    return 0;
}
