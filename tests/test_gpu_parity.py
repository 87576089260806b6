"""GPU parity: the CUDA path, called through the C ABI, against the FP64
oracle on the same seeded inputs, element by element."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1710_08037_gb300 import synth
from tests.helpers import DIAG_TOL, PHASOR_TOL, TOL, ciplv_bound, compare, unpack_phasors

pytestmark = pytest.mark.gpu

PRECISIONS = ["fp32", "bf16x3", "fp16x3"]


@pytest.fixture(scope="module")
def handles():
    import paper_1710_08037_gb300 as plv
    hs = {p: plv.Handle(precision=p) for p in PRECISIONS}
    yield hs
    for h in hs.values():
        h.close()


def _to_np(res):
    return {k: v.double().cpu().numpy() if not v.is_complex()
            else v.cpu().numpy().astype(np.complex128) for k, v in res.items()}


# --- K1: analytic signal + phasors ---------------------------------------------

@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("T", [32, 64, 128, 256, 512, 1024, 2048, 4096, 8192])
def test_analytic_phasors_on_bin_tones(handles, prec, T):
    """Eq. 3-4: on-bin tones have |z| = A exactly, so the phasor must be
    exp(i(2 pi k t/T + th)) to FP32 rounding (no small-|z| samples)."""
    h = handles[prec]
    rng = np.random.default_rng(T)
    N = 7
    t = np.arange(T)
    k = rng.integers(1, T // 2, size=N)
    th = rng.uniform(0, 2 * np.pi, size=N)
    x = np.cos(2 * np.pi * k[:, None] * t / T + th[:, None]) * 3.0
    P = h.plv_analytic(torch.tensor(x[None], device="cuda"))
    got = unpack_phasors(P, prec, 1, N, T)[0]
    ref = np.exp(1j * (2 * np.pi * k[:, None] * t / T + th[:, None]))
    assert np.max(np.abs(got - ref)) < PHASOR_TOL[prec]


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("T", [2, 3, 33, 100, 500, 600, 997, 1000, 2400, 3001, 4097, 8191,
                               9999, 10000, 12288])
def test_analytic_any_length_vs_oracle(handles, prec, T):
    """Eq. 3-4 for lengths that are not powers of two (the circular
    convolution with the periodic Hilbert kernel): against the oracle's
    direct DFT, in z, with zero padding samples."""
    h = handles[prec]
    rng = np.random.default_rng(T)
    B, N = 1, 3
    x = rng.standard_normal((B, N, T))
    P = h.plv_analytic(torch.tensor(x, device="cuda", dtype=torch.float32))
    got = unpack_phasors(P, prec, B, N, T)
    z = oracle.analytic(x.astype(np.float32).astype(np.float64))
    ref = z / np.abs(z)
    rms = np.sqrt(np.mean(np.abs(z) ** 2))
    err_z = np.abs(got - ref) * np.abs(z)
    assert err_z.max() < max(2e-5, PHASOR_TOL[prec]) * rms, err_z.max() / rms
    ld = ((T + 31) // 32) * 32
    if prec == "fp32" and ld > T:
        pad = P[: B * N * 2 * ld].view(B, N, 2, ld)[..., T:]
        assert torch.all(pad == 0)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_end_to_end_any_length(handles, prec):
    """Whole path at T = 1000 and T = 2500 (ragged N) against the oracle."""
    h = handles[prec]
    for (N, T) in ((70, 1000), (129, 2500)):
        x = synth.bandlimited(1, N, T, seed=T, device="cuda")
        res = _to_np(h.connectivity(x, C=True))
        ref = oracle.connectivity(x[0].double().cpu().numpy())
        gpu = {k: res[k][0] for k in ("plv", "iplv", "ciplv")}
        compare(gpu, ref, TOL[prec])


@pytest.mark.parametrize("prec", PRECISIONS)
def test_analytic_phasors_random_vs_oracle(handles, prec):
    """Eq. 3-4 on white noise against the oracle's direct DFT: phasor error
    scales like (FFT error)/|z|, so compare where |z| is not tiny."""
    h = handles[prec]
    rng = np.random.default_rng(3)
    B, N, T = 2, 5, 1024
    x = rng.standard_normal((B, N, T))
    P = h.plv_analytic(torch.tensor(x, device="cuda", dtype=torch.float32))
    got = unpack_phasors(P, prec, B, N, T)
    z = oracle.analytic(x.astype(np.float32).astype(np.float64))
    ref = z / np.abs(z)
    # the phasor error is the FFT's error in z divided by |z|: compare in z
    rms = np.sqrt(np.mean(np.abs(z) ** 2))
    err_z = np.abs(got - ref) * np.abs(z)
    assert err_z.max() < max(1e-5, PHASOR_TOL[prec]) * rms
    assert np.abs(np.abs(got) - 1).max() < max(1e-6, PHASOR_TOL[prec])


# --- K2/K3: Gram + read-outs ---------------------------------------------------

@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("B,N,T", [(1, 1, 32), (1, 3, 64), (2, 67, 96),
                                   (1, 129, 256), (3, 200, 160),
                                   (1, 256, 1000)])
def test_gram_parity_given_analytic_signal(handles, prec, B, N, T):
    """Eq. 7, 13, 14 from the oracle's own analytic signal (normalised on
    the GPU by plv_normalize): ragged N (partial tiles), ragged T (padding)."""
    h = handles[prec]
    rng = np.random.default_rng(N * 1000 + T)
    x = rng.standard_normal((B, N, T))
    z = oracle.analytic(x)
    P = h.plv_normalize(torch.tensor(z, device="cuda"))
    res = _to_np(h.plv_gram(P, B, N, T, C=True))
    for e in range(B):
        ref = oracle.pairwise(z[e])
        gpu = {k: res[k][e] for k in ("plv", "iplv", "ciplv")}
        compare(gpu, ref, TOL[prec])
        assert np.max(np.abs(res["C"][e] - ref["c"])) < TOL[prec]


@pytest.mark.parametrize("prec", PRECISIONS)
def test_end_to_end_tones_workload(handles, prec):
    """The small parity workload (64 channels, T = 2048, FP64 input): whole
    path x -> PLV / iPLV / ciPLV against the oracle's pairwise loop."""
    h = handles[prec]
    x, meta = synth.tones(seed=1001)
    res = _to_np(h.connectivity(torch.tensor(x, device="cuda"), C=True,
                                diag=True))
    ref = oracle.connectivity(x[0])
    gpu = {k: res[k][0] for k in ("plv", "iplv", "ciplv")}
    errs = compare(gpu, ref, TOL[prec])
    assert res["diag"][0] < DIAG_TOL[prec]
    # the closed-form structure survives: coupled pairs lock, sign of lead
    for (a, b), d in zip(meta["pairs"], meta["deltas"]):
        if abs(math.sin(d)) > 0.2:
            assert gpu["ciplv"][a, b] > 0 and gpu["ciplv"][b, a] < 0
    print(prec, errs)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_symmetry_is_exact(handles, prec):
    """The lower triangle is a mirror of the upper one, bit for bit."""
    h = handles[prec]
    x = synth.bandlimited(2, 300, 512, seed=17, device="cuda")
    res = h.connectivity(x, C=True)
    assert torch.equal(res["plv"], res["plv"].transpose(1, 2))
    assert torch.equal(res["iplv"], res["iplv"].transpose(1, 2))
    assert torch.equal(res["ciplv"], -res["ciplv"].transpose(1, 2))
    assert torch.equal(res["C"], res["C"].transpose(1, 2).conj())
    d = torch.diagonal(res["ciplv"], dim1=1, dim2=2)
    assert torch.all(d == 0)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_metrics_kernel_matches_fused_epilogue(handles, prec):
    """plv_metrics on the stored C gives the fused epilogue's bits."""
    h = handles[prec]
    x = synth.bandlimited(1, 130, 256, seed=2, device="cuda")
    res = h.connectivity(x, C=True)
    m = h.plv_metrics(res["C"])
    for k in ("plv", "iplv", "ciplv"):
        assert torch.equal(m[k], res[k]), k


@pytest.mark.parametrize("prec", PRECISIONS)
def test_ciplv_near_zero_lag_tones(handles, prec):
    """Eq. 14 where it is ill-conditioned: on-bin tone pairs at lags of
    1e-1, 1e-2 and 3e-3 rad (1 - Re^2 = sin^2 lag down to ~1e-5), whole path
    from x, ciPLV element by element against the oracle within the
    first-order conditioned bound of the path's tolerance; the closed form
    (Section II.C: a pure lag gives ciPLV = sign(sin lag)) must survive where
    the bound is below 1."""
    h = handles[prec]
    T, k0 = 2048, 40
    lags = [1e-1, -1e-1, 1e-2, -1e-2, 3e-3, -3e-3]
    t = np.arange(T)
    rows, pairs = [], []
    rng = np.random.default_rng(7)
    for lag in lags:
        th = rng.uniform(0, 2 * np.pi)
        rows.append(np.cos(2 * np.pi * k0 * t / T + th))
        rows.append(np.cos(2 * np.pi * k0 * t / T + th - lag))
        pairs.append((len(rows) - 2, len(rows) - 1, lag))
    x = np.stack(rows)[None]
    res = _to_np(h.connectivity(torch.tensor(x, device="cuda"), C=True))
    ref = oracle.connectivity(x[0])
    gpu = {k: res[k][0] for k in ("plv", "iplv", "ciplv")}
    compare(gpu, ref, TOL[prec])
    for a, b, lag in pairs:
        # oracle: the closed form, to FP64 rounding amplified by 1/|sin lag|
        assert abs(ref["ciplv"][a, b] - math.copysign(1.0, math.sin(lag))) < 1e-9 / abs(lag)
        bound = float(ciplv_bound(np.asarray(ref["c"][a, b]), TOL[prec]))
        if bound < 0.5:
            assert np.sign(gpu["ciplv"][a, b]) == np.sign(math.sin(lag))
            assert np.sign(gpu["ciplv"][b, a]) == -np.sign(math.sin(lag))


@pytest.mark.parametrize("prec", PRECISIONS)
def test_ciplv_denominator_near_unit_real_part(handles, prec):
    """Eq. 14's denominator (1 - Re)(1 + Re) on given FP32 values of C with
    |Re C| from 0.3 to 1 - 2^-24 (where 1 - Re^2 cancels): ciPLV against the
    FP64 value of the same FP32 inputs to a few ulp (the reciprocal square
    root's error; the denominator itself is the error-free FP32 form), and
    0 where Re^2 >= 1."""
    h = handles[prec]
    n = 64
    rng = np.random.default_rng(11)
    C = (rng.uniform(-0.5, 0.5, (1, n, n)) + 1j * rng.uniform(-0.5, 0.5, (1, n, n)))
    C = C.astype(np.complex64)
    re = np.concatenate([
        np.float32(1.0) - np.float32(2.0 ** -24) * np.arange(1, 9, dtype=np.float32),
        np.float32(1.0) - np.float32(2.0 ** -6) * np.array([0.5, 1.0, 1.5, 2.0], np.float32),
        np.float32(1.0) - np.float32(2.0 ** -12) * np.arange(1, 5, dtype=np.float32),
        np.array([0.3, 0.5, 0.75, 0.9, 1.0, 1.0 + 2 ** -23], np.float32)]).astype(np.float32)
    re = np.concatenate([re, -re])
    im = (rng.uniform(1e-4, 1e-2, re.size) * rng.choice([-1, 1], re.size)).astype(np.float32)
    ii = np.arange(re.size) % n
    jj = (ii + 1 + np.arange(re.size) // n) % n  # off the diagonal
    C[0, ii, jj] = re + 1j * im
    m = h.plv_metrics(torch.tensor(C, device="cuda"))
    got = m["ciplv"][0].double().cpu().numpy()[ii, jj]
    r64, i64 = re.astype(np.float64), im.astype(np.float64)
    d = (1.0 - r64) * (1.0 + r64)
    want = np.where(d > 0, i64 / np.sqrt(np.where(d > 0, d, 1.0)), 0.0)
    rel = np.abs(got - want) / np.maximum(np.abs(want), 1e-30)
    assert np.all(rel[d > 0] < 1e-6), float(rel[d > 0].max())
    assert np.all(got[d <= 0] == 0.0)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_zero_row(handles, prec):
    """|z| = 0 everywhere on one channel: its phasors are 0, PLV row 0."""
    h = handles[prec]
    x = torch.randn(1, 40, 256, device="cuda", dtype=torch.float64)
    x[0, 7] = 0
    res = h.connectivity(x)
    assert torch.all(res["plv"][0, 7] == 0) and torch.all(res["plv"][0, :, 7] == 0)
    assert torch.all(res["ciplv"][0, 7] == 0)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_empty_batch_is_noop(handles, prec):
    h = handles[prec]
    x = torch.empty(0, 4, 64, device="cuda")
    P = h.plv_analytic(x)
    res = h.plv_gram(P, 0, 4, 64)
    assert res["plv"].shape == (0, 4, 4)


def test_invalid_arguments_are_rejected(handles):
    """Host-side validation: nothing is launched, an error status returns."""
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import _lib
    h = handles["fp32"]
    with pytest.raises(plv.PlvError) as ei:
        h.plv_analytic(torch.randn(1, 2, 20000, device="cuda"))  # T too long
    assert ei.value.status == _lib.PLV_ERR_UNSUPPORTED
    x = torch.randn(1, 4, 100, device="cuda")
    P = h.empty_phasors(1, 4, 64)
    rc = h.lib.plv_gram(h.h, None, None, 1, 4, 64, 1, None, None, None, None,
                        None)
    assert rc == _lib.PLV_ERR_INVALID
    rc = h.lib.plv_analytic(h.h, None, x.data_ptr(), 0, 1, 4, 64, 32,
                            P.data_ptr())  # ldx < T
    assert rc == _lib.PLV_ERR_INVALID
    rc = h.lib.plv_gram(h.h, None, P.data_ptr(), 1, 4, 64, 1 << 6, None,
                        None, None, None, None)  # unknown output bit
    assert rc == _lib.PLV_ERR_INVALID
    assert h.plv_sync_status() == 0


# --- full-size workload: sampled outputs + invariants -----------------------

def _sampled_check(h, prec, E, N, T, seed, n_rows=12, n_cols=48, n_ep=2):
    x = synth.bandlimited(E, N, T, seed=seed, device="cuda")
    res = h.connectivity(x, diag=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    eps = TOL[prec]
    worst = {"plv": 0.0, "iplv": 0.0, "ciplv": 0.0}
    for e in rng.choice(E, size=min(n_ep, E), replace=False):
        rows = rng.choice(N, size=n_rows, replace=False)
        cols = rng.choice(N, size=n_cols, replace=False)
        pi = np.repeat(rows, n_cols)
        pj = np.tile(cols, n_rows)
        ref = oracle.connectivity_pairs(x[e].double().cpu().numpy(), pi, pj)
        ii = torch.tensor(pi, device="cuda")
        jj = torch.tensor(pj, device="cuda")
        gpu = {k: res[k][int(e)][ii, jj].double().cpu().numpy()
               for k in ("plv", "iplv", "ciplv")}
        errs = compare(gpu, ref, eps)
        for k in worst:
            worst[k] = max(worst[k], errs[k])
    # invariants on the whole output
    assert float(res["diag"].max()) < DIAG_TOL[prec]
    assert float(res["plv"].max()) <= 1.0 + 1e-5
    assert bool(torch.all(res["iplv"] <= res["plv"] + 1e-6))
    return worst


def test_full_size_fp32_workload_sampled():
    """N = 4096 sources, T = 4096, 30 epochs, band-limited 8-12 Hz with
    coupling and leakage (the FP32 workload), sampled pairs vs the oracle."""
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision="fp32")
    w = _sampled_check(h, "fp32", 30, 4096, 4096, seed=1002)
    print("fp32 full-size worst errors", w)
    h.close()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
def test_full_size_split_workload_sampled(prec):
    """N = 8192 sources, T = 8192, 20 epochs (the split-precision workload),
    sampled pairs vs the oracle plus invariants on the whole output."""
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision=prec)
    w = _sampled_check(h, prec, 20, 8192, 8192, seed=1003, n_rows=8,
                       n_cols=32)
    print(prec, "full-size worst errors", w)
    h.close()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
def test_gram_raster_changes_no_bits(prec):
    """plv_set_gram_raster reorders which CTA computes a tile, never its
    value: outputs are identical for raster widths 1, 3, 16 and the plain
    column-major triangle (width >= row blocks), with ragged N."""
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision=prec)
    x = synth.bandlimited(2, 1100, 512, seed=5, device="cuda")  # 9 row blocks
    P = h.plv_analytic(x)
    ref = None
    for w in (0, 1, 3, 16, 9, 100):
        h.set_gram_raster(w)
        res = h.plv_gram(P, 2, 1100, 512, C=True)
        if ref is None:
            ref = res
            continue
        for k in ("plv", "iplv", "ciplv", "C"):
            assert torch.equal(res[k], ref[k]), (w, k)
    import ctypes
    assert h.lib.plv_set_gram_raster(h.h, -1) != 0
    h.close()
