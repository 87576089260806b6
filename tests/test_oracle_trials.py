"""Pins of the oracle's functions over trials and windows (CPU): the
time-resolved PLV (Eq. 1 / Eq. 8), the DFT at selected bins, coherency
across trials (Eq. 12) and the sliding-window PLV, each against something
other than itself -- the reformulated Gram, closed forms for on-bin tones
and lag changes, the Rayleigh null, numpy's FFT, the tiling identity, and
invariances that a wrong index, sign or normaliser breaks."""
import numpy as np
import pytest

import oracle


def _tones_with_trial_phase(E, N, T, k, seed):
    """On-bin tones cos(2 pi k t / T + theta_n + delta_i): every trial n has
    its own phase theta_n, common to all channels; channel i has delta_i."""
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0, 2 * np.pi, E)
    delta = rng.uniform(0, 2 * np.pi, N)
    t = np.arange(T)
    x = np.cos(2 * np.pi * k * t[None, None, :] / T + theta[:, None, None]
               + delta[None, :, None])
    return x, delta


def test_time_resolved_equals_reformulated_gram_per_sample():
    """Eq. 1 evaluated with phases (atan2 / exp) equals, at every sample t,
    the reformulated Gram of the trial vectors z_i(t, .) (Eq. 8 is Eq. 5-7
    with the trials as the summation index), a zero sample included."""
    rng = np.random.default_rng(11)
    E, N, T = 9, 5, 12
    z = rng.standard_normal((E, N, T)) + 1j * rng.standard_normal((E, N, T))
    z[3, 2, 4] = 0.0
    r = oracle.time_resolved(z, 1, 10)
    for l in range(10):
        g = oracle.gram_direct(z[:, :, 1 + l].T)
        assert np.allclose(r["c"][l], g, atol=1e-13, rtol=0)


def test_time_resolved_tones_closed_form():
    """Trials of on-bin tones with a common per-trial phase: the phase
    difference of i and j is delta_i - delta_j at every sample and trial, so
    PLV(t) = 1, iPLV(t) = |sin(delta_i - delta_j)|, ciPLV(t) = sign of it."""
    E, N, T, k = 7, 6, 64, 5
    x, delta = _tones_with_trial_phase(E, N, T, k, seed=3)
    z = oracle.analytic(x)
    r = oracle.time_resolved(z, 0, T)
    d = delta[:, None] - delta[None, :]
    off = ~np.eye(N, dtype=bool)
    assert np.allclose(r["plv"], 1.0, atol=1e-10)
    assert np.allclose(r["iplv"][:, off], np.abs(np.sin(d))[off], atol=1e-10)
    ok = off & (np.abs(np.cos(d)) < 0.999)
    assert np.allclose(r["ciplv"][:, ok], np.sign(np.sin(d))[ok], atol=1e-6)
    assert np.allclose(np.angle(r["c"][:, off]), np.angle(np.exp(1j * d))[off],
                       atol=1e-10)


def test_time_resolved_rayleigh_null():
    """Independent uniform phases in every trial: the mean of PLV(t) over
    pairs and samples is the Rayleigh mean sqrt(pi / (4 E)) (the 1/E
    normaliser over trials, not over samples)."""
    rng = np.random.default_rng(5)
    E, N, T = 48, 8, 40
    z = np.exp(1j * rng.uniform(0, 2 * np.pi, (E, N, T)))
    r = oracle.time_resolved(z, 0, T)
    off = ~np.eye(N, dtype=bool)
    m = r["plv"][:, off].mean()
    assert abs(m - np.sqrt(np.pi / (4 * E))) < 0.01, m


def test_dft_bins_equals_numpy_fft():
    rng = np.random.default_rng(2)
    for T, f0, F in ((37, 3, 9), (64, 0, 33), (100, 40, 20)):
        x = rng.standard_normal((4, T))
        X = oracle.dft_bins(x, f0, F)
        ref = np.fft.fft(x, axis=-1)[:, f0:f0 + F]
        assert np.allclose(X, ref, atol=1e-10 * T, rtol=0)


def test_coherency_of_unit_phasors_is_plv_over_trials():
    """With |X| = 1 everywhere Eq. 12 reduces to the PLV over trials
    (Eq. 11 / Eq. 1): the same complex value as the phase-based oracle."""
    rng = np.random.default_rng(4)
    E, N, L = 10, 5, 6
    X = np.exp(1j * rng.uniform(0, 2 * np.pi, (E, N, L)))
    c = oracle.coherency_trials(X)
    r = oracle.time_resolved(X, 0, L)
    assert np.allclose(c["c"], r["c"], atol=1e-13, rtol=0)


def test_coherency_closed_form_of_a_scaled_copy():
    """X_j = a X_i for a complex constant a: coh_ij = conj(a) / |a|, so the
    coherence is 1 and the imaginary coherency is |Im a| / |a|; the lagged
    coherence is -sign(Im a) (|Re| < 1)."""
    rng = np.random.default_rng(6)
    E, L = 12, 3
    Xi = rng.standard_normal((E, 1, L)) + 1j * rng.standard_normal((E, 1, L))
    a = 0.7 * np.exp(1j * 1.1)
    X = np.concatenate([Xi, a * Xi], axis=1)
    c = oracle.coherency_trials(X)
    assert np.allclose(c["c"][:, 0, 1], np.conj(a) / abs(a), atol=1e-13)
    assert np.allclose(c["coh"][:, 0, 1], 1.0, atol=1e-13)
    assert np.allclose(c["icoh"][:, 0, 1], abs(a.imag) / abs(a), atol=1e-13)
    assert np.allclose(c["lcoh"][:, 0, 1], -np.sign(a.imag), atol=1e-9)


def test_coherency_invariances_and_bounds():
    """Unchanged by a positive per-channel gain and by a per-trial phase
    common to all channels; Hermitian; |coh| <= 1 (Cauchy-Schwarz); unit
    diagonal; a zero channel gives 0."""
    rng = np.random.default_rng(8)
    E, N, L = 15, 6, 4
    X = rng.standard_normal((E, N, L)) + 1j * rng.standard_normal((E, N, L))
    X[:, 5, :] = 0.0
    c = oracle.coherency_trials(X)["c"]
    gain = rng.uniform(0.2, 5.0, (1, N, 1))
    rot = np.exp(1j * rng.uniform(0, 2 * np.pi, (E, 1, L)))
    c2 = oracle.coherency_trials(X * gain * rot)["c"]
    assert np.allclose(c, c2, atol=1e-12, rtol=0)
    assert np.allclose(c, np.conj(np.swapaxes(c, 1, 2)), atol=1e-14)
    assert np.all(np.abs(c) <= 1 + 1e-12)
    assert np.allclose(np.diagonal(c, axis1=1, axis2=2)[:, :5], 1.0, atol=1e-13)
    assert np.all(c[:, 5, :] == 0) and np.all(c[:, :, 5] == 0)
    # amplitude weighting: coherency is not the PLV of the same values
    p = oracle.time_resolved(X[:, :5], 0, L)["c"]
    assert np.abs(c[:, :5, :5] - p).max() > 1e-3


def test_windows_tile_the_whole_signal():
    """Windows that tile [0, T) without overlap: T c_full = sum_w W c_w (the
    per-window normaliser and offsets), for random phases."""
    rng = np.random.default_rng(12)
    N, T, W = 6, 160, 32
    z = rng.standard_normal((N, T)) + 1j * rng.standard_normal((N, T))
    r = oracle.windows(z, 0, W, W, T // W)
    full = oracle.pairwise(z)["c"]
    assert np.allclose(W * r["c"].sum(axis=0), T * full, atol=1e-12)
    one = oracle.windows(z, 0, T, 0, 1)
    assert np.allclose(one["c"][0], full, atol=1e-14)


def test_windows_track_a_lag_change():
    """The lag between two channels switches at T/2: windows inside each half
    give exp(i delta) of that half, a window across the switch the weighted
    mean of the two (closed forms)."""
    T, W = 256, 64
    t = np.arange(T)
    d1, d2 = 0.7, -1.9
    ph = 2 * np.pi * 0.05 * t
    z = np.stack([np.exp(1j * ph), np.exp(1j * (ph - np.where(t < T // 2, d1, d2)))])
    r = oracle.windows(z, 0, W, 32, (T - W) // 32 + 1)
    for w in range(r["c"].shape[0]):
        a = w * 32
        n1 = max(0, min(T // 2, a + W) - a)
        want = (n1 * np.exp(1j * d1) + (W - n1) * np.exp(1j * d2)) / W
        assert abs(r["c"][w, 0, 1] - want) < 1e-12, (w, r["c"][w, 0, 1], want)
