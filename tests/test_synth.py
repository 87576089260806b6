"""The seeded synthetic inputs on CPU: reproducible from their seeds, rows at
unit RMS, power inside the requested band, the Butterworth magnitude-squared
response, and the tones workload's planted structure."""
import numpy as np
import torch

from paper_1710_08037_gb300 import synth


def test_bandlimited_is_reproducible_and_seed_dependent():
    a = synth.bandlimited(2, 16, 1000, seed=11)
    b = synth.bandlimited(2, 16, 1000, seed=11)
    c = synth.bandlimited(2, 16, 1000, seed=12)
    assert torch.equal(a, b)
    assert not torch.equal(a, c)


def test_bandlimited_rows_have_unit_rms_and_power_in_band():
    fs, band, T = 1000.0, (8.0, 12.0), 4096
    x = synth.bandlimited(1, 32, T, seed=3, fs=fs, band=band).double().numpy()[0]
    rms = np.sqrt(np.mean(x ** 2, axis=1))
    assert np.allclose(rms, 1.0, atol=1e-5)
    p = np.abs(np.fft.rfft(x, axis=1)) ** 2
    f = np.fft.rfftfreq(T, d=1.0 / fs)
    inside = (f >= band[0] - 2.0) & (f <= band[1] + 2.0)
    assert p[:, inside].sum() / p.sum() > 0.9


def test_butter_power_is_a_band_pass_magnitude_squared():
    T, fs = 4096, 1000.0
    h2 = synth.butter_power(T, fs, (8.0, 12.0))
    f = np.fft.rfftfreq(T, d=1.0 / fs)
    assert h2.shape == (T // 2 + 1,)
    assert np.all(h2 >= 0.0) and np.all(h2 <= 1.0 + 1e-9)
    assert h2[np.argmin(np.abs(f - 10.0))] > 0.9      # passband
    assert h2[0] < 1e-6 and h2[np.argmin(np.abs(f - 100.0))] < 1e-6  # stopbands


def test_tones_plant_lagged_pairs_and_zero_lag_mixtures():
    x, meta = synth.tones(seed=1001, noise=0.0)
    clean = meta["clean"][0]
    assert x.shape == (1, 64, 2048)
    T, k = 2048, int(round(meta["bin"]))
    assert k == 40  # 10 Hz at fs = 512 Hz, T = 2048: an exact DFT bin
    for (a, b), d in zip(meta["pairs"], meta["deltas"]):
        # channel b is channel a's tone shifted in phase by the planted lag
        za = np.fft.rfft(clean[a])[k]
        zb = np.fft.rfft(clean[b])[k]
        lag = np.angle(za / zb)
        assert abs((lag - d + np.pi) % (2 * np.pi) - np.pi) < 1e-9
    for (m, p, q, al, be) in meta["mixes"]:
        assert np.allclose(clean[m], al * clean[p] + be * clean[q])


def test_pair_mask_excludes_the_diagonal():
    m = synth.random_pair_mask(100, 0.1, seed=1005)
    assert not bool(m.diagonal().any())
    frac = float(m.sum()) / (100 * 99)
    assert 0.07 < frac < 0.13
    assert torch.equal(m, synth.random_pair_mask(100, 0.1, seed=1005))
