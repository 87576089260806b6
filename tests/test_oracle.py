"""Pins for the FP64 oracle, against things other than the oracle itself:
a library analytic signal, closed forms, brute force and statistics.

Each test names the passage of the paper it pins.  CPU only.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import backward as obw
from paper_1710_08037_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- Eq. 3: analytic signal -------------------------------------------------

@pytest.mark.parametrize("T", [1, 2, 3, 4, 5, 8, 16, 17, 31, 64, 100, 127,
                               128, 256, 500])
def test_analytic_matches_scipy_hilbert(T):
    """Eq. 3: the direct-DFT analytic signal equals scipy's FFT-based
    discrete analytic signal (same mask h) for even and odd T."""
    from scipy.signal import hilbert
    rng = np.random.default_rng(T)
    x = rng.standard_normal((3, T))
    z = oracle.analytic(x)
    ref = hilbert(x, axis=-1)
    assert np.max(np.abs(z - ref)) < 1e-11 * max(1.0, T / 64)


@pytest.mark.parametrize("T,k", [(64, 1), (64, 5), (64, 31), (2048, 40),
                                 (100, 7), (127, 63), (500, 123)])
def test_analytic_on_bin_tone(T, k):
    """Eq. 3 / Eq. 10: for an on-bin tone A cos(2 pi k t/T + th), 0<k<T/2,
    the analytic signal is exactly A exp(i(2 pi k t/T + th))."""
    t = np.arange(T)
    th = 0.3 + k
    x = 1.7 * np.cos(2 * np.pi * k * t / T + th)
    z = oracle.analytic(x[None])[0]
    ref = 1.7 * np.exp(1j * (2 * np.pi * k * t / T + th))
    assert np.max(np.abs(z - ref)) < 1e-11


def test_analytic_dc_and_nyquist_map_to_themselves():
    """h[0] = h[T/2] = 1: a constant and an alternating sequence have zero
    Hilbert transform, so z = x."""
    T = 64
    x = np.stack([np.full(T, 2.5), (-1.0) ** np.arange(T)])
    z = oracle.analytic(x)
    assert np.max(np.abs(z - x)) < 1e-12


def test_analytic_real_part_is_input():
    """h[k] + h[-k] = 2 for every k, so Re z = x for any real x."""
    rng = np.random.default_rng(5)
    for T in (7, 64, 99):
        x = rng.standard_normal((4, T))
        z = oracle.analytic(x)
        assert np.max(np.abs(z.real - x)) < 1e-12


# --- Eq. 2 and Eq. 5-7: pairwise definition vs reformulation -----------------

def test_pairwise_equals_reformulated_gram():
    """Eq. 5-7: (1/T) sum exp(i(phi_i - phi_j)) equals the normalised
    Hermitian product, by brute force on tiny inputs."""
    rng = np.random.default_rng(11)
    for N, T in ((1, 1), (3, 5), (7, 33), (16, 256)):
        z = rng.standard_normal((N, T)) + 1j * rng.standard_normal((N, T))
        c1 = oracle.pairwise(z)["c"]
        c2 = oracle.gram_direct(z)
        assert np.max(np.abs(c1 - c2)) < 1e-12


def test_pairwise_equals_numpy_matmul_of_phasors():
    """Eq. 7 written with a library matmul: C = P P^H / T."""
    rng = np.random.default_rng(12)
    z = rng.standard_normal((9, 40)) + 1j * rng.standard_normal((9, 40))
    P = z / np.abs(z)
    C = P @ P.conj().T / 40
    assert np.max(np.abs(oracle.pairwise(z)["c"] - C)) < 1e-12


def test_lagged_tones_golden():
    """Section II.C (Eq. 13, 14): golden closed-form values for two on-bin
    tones with a constant lag, through the whole oracle path."""
    rows = np.loadtxt(os.path.join(GOLDEN, "lagged_tones.txt"))
    T, k = 256, 9
    t = np.arange(T)
    for delta, plv, iplv, ci_ij, ci_ji in rows:
        x = np.stack([np.cos(2 * np.pi * k * t / T + 0.4),
                      np.cos(2 * np.pi * k * t / T + 0.4 - delta)])
        out = oracle.connectivity(x)
        assert abs(out["plv"][0, 1] - plv) < 1e-10
        assert abs(out["iplv"][0, 1] - iplv) < 1e-10
        assert abs(out["ciplv"][0, 1] - ci_ij) < 1e-8
        assert abs(out["ciplv"][1, 0] - ci_ji) < 1e-8
        assert abs(out["plv"][1, 0] - plv) < 1e-10


def test_tones_workload_closed_form():
    """The noise-free parity workload: every coupled pair has PLV = 1,
    iPLV = |sin delta| and ciPLV = +1 (leader first), -1 transposed."""
    _, meta = synth.tones(seed=1001, noise=0.0)
    out = oracle.connectivity(meta["clean"][0])
    for (a, b), d in zip(meta["pairs"], meta["deltas"]):
        assert abs(out["plv"][a, b] - 1.0) < 1e-10
        assert abs(out["iplv"][a, b] - abs(math.sin(d))) < 1e-10
        if abs(math.sin(d)) > 1e-3:
            assert abs(out["ciplv"][a, b] - 1.0) < 1e-6
            assert abs(out["ciplv"][b, a] + 1.0) < 1e-6


def test_zero_lag_copy_has_no_imaginary_part():
    """Section II.C: an instantaneous (zero-lag) copy, here with a sign flip,
    has Im c = 0, so iPLV = ciPLV = 0 while PLV = 1."""
    rng = np.random.default_rng(3)
    x0 = rng.standard_normal(128)
    x = np.stack([x0, -0.5 * x0, 2.0 * x0])
    out = oracle.connectivity(x)
    assert np.allclose(out["plv"], 1.0, atol=1e-12)
    assert np.max(np.abs(out["iplv"])) < 1e-12
    assert np.max(np.abs(out["ciplv"])) < 1e-12
    assert abs(out["c"][0, 1].real + 1.0) < 1e-12


def test_symmetry_and_bounds():
    """c_ji = conj(c_ij) (Eq. 6): PLV and iPLV symmetric, ciPLV
    antisymmetric; 0 <= iPLV <= PLV <= 1; diagonal PLV 1, iPLV = ciPLV = 0."""
    x, _ = synth.tones(seed=1001)
    out = oracle.connectivity(x[0])
    c = out["c"]
    assert np.max(np.abs(c - c.conj().T)) < 1e-13
    assert np.max(np.abs(out["plv"] - out["plv"].T)) < 1e-13
    assert np.max(np.abs(out["ciplv"] + out["ciplv"].T)) < 1e-12
    assert out["plv"].max() <= 1.0 + 1e-12
    assert np.all(out["iplv"] <= out["plv"] + 1e-15)
    assert np.allclose(np.diag(out["plv"]), 1.0, atol=1e-12)
    assert np.all(np.diag(out["iplv"]) == 0.0)
    assert np.all(np.diag(out["ciplv"]) == 0.0)


def test_time_shift_invariance():
    """Eq. 2 averages over time: a common circular shift leaves c
    unchanged."""
    x, _ = synth.tones(seed=7, N=12, T=256, n_pairs=3, n_mix=2)
    c0 = oracle.connectivity(x[0])["c"]
    c1 = oracle.connectivity(np.roll(x[0], 37, axis=-1))["c"]
    assert np.max(np.abs(c0 - c1)) < 1e-12


def test_rayleigh_null_mean():
    """Independent uniform phases: E[PLV] = sqrt(pi/(4T)) (Rayleigh mean of
    |mean of T unit phasors|), sd sqrt((4-pi)/(4T)).  Pins the 1/T factor."""
    N, T = 64, 2048
    z = synth.uniform_phases(N, T, seed=99)
    plv = oracle.pairwise(z)["plv"]
    iu = np.triu_indices(N, 1)
    vals = plv[iu]
    mean = math.sqrt(math.pi / (4 * T))
    se = math.sqrt((4 - math.pi) / (4 * T)) / math.sqrt(vals.size)
    assert abs(vals.mean() - mean) < 5 * se


def test_zero_row_contributes_nothing():
    """Eq. 4 divides by |z|: a sample without amplitude has no phase; its
    phasor is taken as 0, so an all-zero channel has PLV 0 with everyone."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((4, 64))
    x[2] = 0.0
    out = oracle.connectivity(x)
    assert np.all(out["plv"][2] == 0.0) and np.all(out["plv"][:, 2] == 0.0)
    assert out["plv"][1, 1] == pytest.approx(1.0)


def test_metrics_closed_forms():
    """Eq. 7, 13, 14 on hand-computed values."""
    c = np.array([0.6 + 0.8j, 0.3 - 0.4j, 1.0 + 0j, -1.0 + 0j, 0j])
    m = oracle.metrics(c)
    assert np.allclose(m["plv"], [1.0, 0.5, 1.0, 1.0, 0.0], atol=1e-15)
    assert np.allclose(m["iplv"], [0.8, 0.4, 0.0, 0.0, 0.0], atol=1e-15)
    assert np.allclose(m["ciplv"], [1.0, -0.4 / math.sqrt(0.91), 0.0, 0.0,
                                    0.0], atol=1e-15)


def test_single_source_mixture_ciplv_small():
    """Section II.C / Eq. 16: a zero-lag mixture of one band-limited source
    with independent noise has ciPLV ~ 0 (statistical: a few / sqrt(T_eff)),
    while a lagged copy keeps |ciPLV| large."""
    import torch
    src = synth.bandlimited(1, 3, 4096, seed=5, coupled_frac=0.0,
                            leak_frac=0.0, dtype=torch.float64)[0].numpy()
    x = np.stack([src[0], 0.7 * src[0] + 0.5 * src[1],
                  np.roll(src[0], 25)])
    out = oracle.connectivity(x)
    teff = 2 * 4.0 * 4096 / 1000.0  # 2 * bandwidth * T / fs (Section III.B)
    assert abs(out["ciplv"][0, 1]) < 4.0 / math.sqrt(teff)
    assert out["plv"][0, 1] > 0.5
    assert abs(out["ciplv"][0, 2]) > 0.5


# --- gradient references pin each other --------------------------------------

def test_backward_references_agree():
    """Central finite differences of the FP64 oracle vs FP64 autograd through
    plain torch ops, for a loss mixing all three metrics."""
    rng = np.random.default_rng(21)
    N, T = 5, 48
    x = rng.standard_normal((N, T))
    g1 = rng.standard_normal((N, N))
    g2 = rng.standard_normal((N, N))
    g3 = rng.standard_normal((N, N))
    np.fill_diagonal(g3, 0.0)
    np.fill_diagonal(g2, 0.0)
    gt = obw.torch_grad(x, g1, g2, g3).reshape(-1)
    ent = rng.choice(N * T, size=40, replace=False)
    gf = obw.fd_grad(x, g1, g2, g3, entries=ent)
    scale = np.max(np.abs(gt))
    assert np.max(np.abs(gf - gt[ent])) < 1e-6 * max(1.0, scale)


def test_torch_forward_matches_oracle():
    """The autograd reference's forward is the same function as the
    oracle's."""
    import torch
    rng = np.random.default_rng(22)
    x = rng.standard_normal((6, 50))
    C, plv, iplv, ciplv = obw.torch_forward(torch.tensor(x))
    out = oracle.connectivity(x)
    assert np.max(np.abs(C.numpy() - out["c"])) < 1e-12
    assert np.max(np.abs(ciplv.numpy() - out["ciplv"])) < 1e-10
