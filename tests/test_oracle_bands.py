"""Pins of the oracle's band-limited analytic signal (CPU): the band-pass
and the analytic mask applied in one transform (the band-pass then analytic
signal of Section III.A), against scipy's Hilbert transform of the
band-passed signal, on-bin tone closed forms and linearity."""
import numpy as np
import pytest

import oracle


def _full_mask(band, T):
    """The real, even mask on all T bins whose half is ``band``."""
    k = np.arange(T)
    return band[np.minimum(k, T - k)]


@pytest.mark.parametrize("T", [64, 65, 100])
def test_band_all_ones_is_the_analytic_signal(T):
    x = np.random.default_rng(T).standard_normal((3, T))
    assert np.allclose(oracle.analytic_band(x, np.ones(T // 2 + 1)), oracle.analytic(x),
                       atol=1e-12)


@pytest.mark.parametrize("T", [64, 97, 128])
def test_band_equals_scipy_hilbert_of_the_band_passed_signal(T):
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(T + 1)
    x = rng.standard_normal((4, T))
    band = rng.uniform(0.0, 1.0, T // 2 + 1)
    u = np.fft.ifft(np.fft.fft(x, axis=-1) * _full_mask(band, T), axis=-1).real
    ref = scipy_signal.hilbert(u, axis=-1)
    assert np.allclose(oracle.analytic_band(x, band), ref, atol=1e-11)


def test_band_selects_one_on_bin_tone():
    """Two on-bin tones; a mask passing only the first leaves exactly its
    analytic signal exp(i (2 pi k1 t / T + theta1))."""
    T, k1, k2 = 128, 9, 23
    t = np.arange(T)
    x = np.cos(2 * np.pi * k1 * t / T + 0.4) + 0.8 * np.cos(2 * np.pi * k2 * t / T - 1.3)
    band = np.zeros(T // 2 + 1)
    band[5:15] = 1.0
    z = oracle.analytic_band(x[None], band)[0]
    assert np.allclose(z, np.exp(1j * (2 * np.pi * k1 * t / T + 0.4)), atol=1e-12)


def test_band_is_linear_in_the_mask():
    x = np.random.default_rng(3).standard_normal((2, 80))
    b1 = np.random.default_rng(4).uniform(0, 1, 41)
    b2 = np.random.default_rng(5).uniform(0, 1, 41)
    lhs = oracle.analytic_band(x, 0.5 * b1 + 2.0 * b2)
    rhs = 0.5 * oracle.analytic_band(x, b1) + 2.0 * oracle.analytic_band(x, b2)
    assert np.allclose(lhs, rhs, atol=1e-12)
