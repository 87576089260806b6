"""Seeded synthetic inputs shaped like the paper's workloads.

This module only makes input signals.  It holds none of the connectivity
arithmetic (no analytic signal, no normalisation, no Gram, no read-outs), so
both the CUDA path and the FP64 oracle can consume what it produces.

The paper measures on resting-state MEG source-space data (Section III.A:
thousands of sources, 1000 Hz, 4 s epochs, alpha band 8-12 Hz) that is not
available here; these generators stand in for it with the same shapes and a
known connectivity structure:

* ``tones``: the small parity workload -- 64 channels of 10 Hz sinusoids at
  fs = 512 Hz (on DFT bin 40 for T = 2048), 16 pairs coupled at a fixed lag,
  8 zero-lag linear mixtures of other channels (the volume-conduction model
  of Section III.C, Eq. 16), 24 independent channels, plus Gaussian noise.
* ``bandlimited``: source-space-like data -- white Gaussian noise band-passed
  (zero-phase 4th-order Butterworth, applied as its squared magnitude on the
  periodic DFT grid), a fraction of channel pairs coupled at random nonzero
  lags (circular shift), a fraction of channels replaced by zero-lag leakage
  mixtures of their index neighbours, and every row rescaled to unit RMS.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def tones(seed: int = 1001, N: int = 64, T: int = 2048, fs: float = 512.0,
          f0: float = 10.0, noise: float = 0.5, n_pairs: int = 16,
          n_mix: int = 8):
    """Parity workload of lagged / mixed sinusoids (FP64, one epoch).

    Channel layout: pairs (2p, 2p+1) for p < n_pairs, with channel 2p+1 the
    sinusoid of channel 2p delayed by a phase lag delta_p ~ U[0, pi); then
    ``n_mix`` zero-lag mixtures alpha x_p + beta x_q (alpha, beta ~
    U(0.3, 0.8), p, q drawn from the non-mixture channels); the rest are
    independent sinusoids.  Every phase offset is U[0, 2 pi).

    Returns ``(x, meta)`` with x float64 (1, N, T) including the noise,
    ``meta['clean']`` the noise-free signals, and the structure.
    """
    rng = np.random.default_rng(seed)
    t = np.arange(T) / fs
    w = 2.0 * np.pi * f0
    clean = np.zeros((N, T))
    theta = rng.uniform(0.0, 2.0 * np.pi, size=N)
    deltas = rng.uniform(0.0, np.pi, size=n_pairs)
    for p in range(n_pairs):
        a, b = 2 * p, 2 * p + 1
        clean[a] = np.cos(w * t + theta[a])
        clean[b] = np.cos(w * t + theta[a] - deltas[p])
    mix0 = 2 * n_pairs
    indep = list(range(mix0 + n_mix, N))
    for c in indep:
        clean[c] = np.cos(w * t + theta[c])
    pool = np.array(list(range(mix0)) + indep)
    mixes = []
    for m in range(n_mix):
        p, q = rng.choice(pool, size=2, replace=False)
        al, be = rng.uniform(0.3, 0.8, size=2)
        clean[mix0 + m] = al * clean[p] + be * clean[q]
        mixes.append((mix0 + m, int(p), int(q), float(al), float(be)))
    x = clean + noise * rng.standard_normal((N, T))
    meta = {"clean": clean[None], "pairs": [(2 * p, 2 * p + 1) for p in
                                            range(n_pairs)],
            "deltas": deltas, "mixes": mixes, "fs": fs, "f0": f0,
            "bin": f0 * T / fs}
    return x[None], meta


def butter_power(T: int, fs: float, band, order: int = 4) -> np.ndarray:
    """Squared magnitude |H(f)|^2 of a digital Butterworth band-pass of the
    given order on the rfft grid of length T (a zero-phase forward-backward
    filter has exactly this response)."""
    from scipy.signal import butter, sosfreqz
    sos = butter(order, list(band), btype="bandpass", fs=fs, output="sos")
    f = np.fft.rfftfreq(T, d=1.0 / fs)
    _, h = sosfreqz(sos, worN=f, fs=fs)
    return np.abs(h) ** 2


def bandlimited(E: int, N: int, T: int, seed: int, fs: float = 1000.0,
                band=(8.0, 12.0), coupled_frac: float = 0.05,
                lag_ms=(5.0, 40.0), kappa=(0.3, 0.8), leak_frac: float = 0.2,
                leak_w=(0.3, 0.8), device="cpu",
                dtype=torch.float32) -> torch.Tensor:
    """Band-limited source-space-like signals, shape (E, N, T).

    Structure parameters (pairs, lags, gains, leakage channels and weights)
    come from a CPU generator seeded with ``seed`` and are identical on every
    device; the white noise comes from a generator on ``device`` seeded with
    ``seed + 1``.  Each coupled pair is directed (driver chosen at random) and
    adds kappa * driver(t - tau) to the driven channel, all contributions
    taken from the uncoupled signals.  Leakage mixes a channel with the mean
    of its two index neighbours, x_m <- (1 - w) x_m + w (x_{m-1} + x_{m+1})/2,
    from the pre-leakage signals.
    """
    dev = torch.device(device)
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    gd = torch.Generator(device=dev).manual_seed(int(seed) + 1)
    out = torch.empty((E, N, T), dtype=dtype, device=dev)
    if E == 0 or N == 0 or T == 0:
        return out
    H2 = torch.as_tensor(butter_power(T, fs, band), dtype=torch.float32,
                         device=dev)
    # structure: coupled pairs grouped by lag, so each lag is one sparse matmul
    lags = {}
    if coupled_frac > 0 and N > 1:
        iu = torch.triu_indices(N, N, offset=1)
        sel = torch.rand(iu.shape[1], generator=g) < coupled_frac
        pi, pj = iu[0][sel], iu[1][sel]
        flip = torch.rand(pi.shape[0], generator=g) < 0.5
        src = torch.where(flip, pj, pi)
        dst = torch.where(flip, pi, pj)
        kap = kappa[0] + (kappa[1] - kappa[0]) * torch.rand(
            pi.shape[0], generator=g, dtype=torch.float64)
        lo = int(round(lag_ms[0] * fs / 1000.0))
        hi = int(round(lag_ms[1] * fs / 1000.0))
        tau = torch.randint(lo, hi + 1, (pi.shape[0],), generator=g)
        for L in torch.unique(tau).tolist():
            m = tau == L
            idx = torch.stack([dst[m], src[m]])
            K = torch.sparse_coo_tensor(idx, kap[m].to(torch.float32),
                                        (N, N)).coalesce().to(dev)
            lags[int(L)] = K
    nleak = int(round(leak_frac * N)) if N > 2 else 0
    leak_ch = torch.randperm(N, generator=g)[:nleak].to(dev)
    leak_wt = (leak_w[0] + (leak_w[1] - leak_w[0]) *
               torch.rand(nleak, generator=g)).to(torch.float32).to(dev)
    for e in range(E):
        w = torch.randn((N, T), generator=gd, device=dev, dtype=torch.float32)
        x = torch.fft.irfft(torch.fft.rfft(w, dim=-1) * H2, n=T, dim=-1)
        y = x.clone()
        for L, K in lags.items():
            y += torch.sparse.mm(K, torch.roll(x, shifts=L, dims=-1))
        if nleak:
            nb = 0.5 * (torch.roll(y, 1, dims=0) + torch.roll(y, -1, dims=0))
            ww = leak_wt[:, None]
            y[leak_ch] = (1.0 - ww) * y[leak_ch] + ww * nb[leak_ch]
        rms = torch.sqrt(torch.mean(y * y, dim=-1, keepdim=True))
        y = y / torch.where(rms > 0, rms, torch.ones_like(rms))
        out[e] = y.to(dtype)
    return out


def random_pair_mask(N: int, frac: float, seed: int, device="cpu"):
    """Seeded boolean (N, N) mask selecting ``frac`` of the ordered pairs
    i != j (the differentiable-loss workload's pair mask)."""
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    m = torch.rand((N, N), generator=g) < frac
    m.fill_diagonal_(False)
    return m.to(device)


def uniform_phases(N: int, T: int, seed: int) -> np.ndarray:
    """Unit phasors with i.i.d. uniform phases, (N, T) complex128: the null
    model whose expected PLV is the Rayleigh mean sqrt(pi / (4 T))."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0.0, 2.0 * math.pi, size=(N, T))
    return np.exp(1j * ph)
