"""The multi-band transform through the C ABI (plv_analytic_bands): band-pass
and analytic signal from one forward FFT per row pair, against the oracle's
band-limited analytic signal (direct DFT, FP64), for every operand
precision, and the whole path to the Gram per band."""
import numpy as np
import pytest
import torch

import oracle
from paper_1710_08037_gb300 import PlvError, synth
from tests.helpers import PHASOR_TOL, TOL, compare, unpack_phasors

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "bf16x3", "fp16x3"]
BANDS = [(4.0, 8.0), (8.0, 12.0), (13.0, 30.0), (30.0, 45.0), (55.0, 80.0)]


@pytest.fixture(scope="module")
def handles():
    import paper_1710_08037_gb300 as plv
    hs = {p: plv.Handle(precision=p) for p in PRECS}
    yield hs
    for h in hs.values():
        h.close()


def _masks(T, fs=1000.0):
    return np.stack([synth.butter_power(T, fs, b) for b in BANDS]).astype(np.float32)


# power-of-two T from 128 to 8192 take the two-rows-per-transform kernel;
# every other T up to 12288 the any-length engine (transform lengths M =
# 128, 2048, 6144, 10240, 20480, 24576 across its four thread classes)
SHAPES = [(1, 7, 128), (2, 33, 1024), (1, 130, 4096), (1, 3, 8192),
          (2, 5, 64), (1, 9, 1000), (1, 6, 3001), (2, 3, 4097), (1, 4, 10000),
          (1, 2, 12288), (1, 131, 600), (1, 1, 3)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("B,N,T", SHAPES)
def test_bands_vs_oracle(handles, prec, B, N, T):
    """Each band's phasors against z / |z| of the oracle's band-limited
    analytic signal, compared in z (a phasor's error is the transform's
    error in z over |z|); ragged N, odd rows, the shortest and longest T."""
    h = handles[prec]
    x = synth.bandlimited(B, N, T, seed=T + N, band=(2.0, 120.0)).double().numpy()
    masks = _masks(T)
    P = h.plv_analytic_bands(torch.tensor(x, device="cuda", dtype=torch.float32),
                             torch.tensor(masks))
    torch.cuda.synchronize()
    xf = x.astype(np.float32).astype(np.float64)
    xrms = np.sqrt(np.mean(xf ** 2))
    for b in range(len(BANDS)):
        got = unpack_phasors(P[b].view(torch.float32), prec, B, N, T)
        z = oracle.analytic_band(xf, masks[b].astype(np.float64))
        a = np.abs(z)
        ref = np.where(a > 0, z / np.where(a > 0, a, 1), 0)
        rms = np.sqrt(np.mean(a ** 2))
        if rms < 1e-5 * xrms:
            # no power in the band above the transform's FP32 rounding (a
            # 3-sample row has no bin in 4-8 Hz): the phase is noise, so only
            # check that every phasor is zero or of unit modulus
            g = np.abs(got)
            assert np.all((g < 1e-6) | (np.abs(g - 1) < 1e-3)), b
            continue
        err_z = np.abs(got - ref) * a
        assert err_z.max() < max(1e-5, PHASOR_TOL[prec]) * rms, (b, err_z.max() / rms)


@pytest.mark.parametrize("prec", PRECS)
def test_bands_then_gram_vs_oracle(handles, prec):
    """Per band: phasors from the fused transform, then plv_gram, against
    the oracle's band-limited analytic signal and pairwise definition."""
    h = handles[prec]
    E, N, T = 2, 60, 2048
    x = synth.bandlimited(E, N, T, seed=31, band=(2.0, 120.0)).double().numpy()
    masks = _masks(T)
    P = h.plv_analytic_bands(torch.tensor(x, device="cuda", dtype=torch.float32),
                             torch.tensor(masks))
    xf = x.astype(np.float32).astype(np.float64)
    for b in (1, 3):
        res = h.plv_gram(P[b].view(torch.float32), E, N, T)
        torch.cuda.synchronize()
        for e in range(E):
            z = oracle.analytic_band(xf[e], masks[b].astype(np.float64))
            ref = oracle.pairwise(z)
            compare({k: res[k][e].double().cpu().numpy() for k in ("plv", "iplv", "ciplv")},
                    ref, TOL[prec])


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_bands_any_length_then_gram_vs_oracle(handles, prec):
    """Any-length bands (T = 2500) through plv_gram, against the oracle; a
    second call with other masks (a new kernel set) and a repeat of the
    first (from the handle's cache) give the same phasors as fresh ones."""
    h = handles[prec]
    E, N, T = 2, 40, 2500
    x = synth.bandlimited(E, N, T, seed=41, band=(2.0, 120.0)).double().numpy()
    xt = torch.tensor(x, device="cuda", dtype=torch.float32)
    masks = _masks(T)
    P = h.plv_analytic_bands(xt, torch.tensor(masks))
    xf = x.astype(np.float32).astype(np.float64)
    for b in (0, 2):
        res = h.plv_gram(P[b].view(torch.float32), E, N, T)
        torch.cuda.synchronize()
        for e in range(E):
            z = oracle.analytic_band(xf[e], masks[b].astype(np.float64))
            compare({k: res[k][e].double().cpu().numpy() for k in ("plv", "iplv", "ciplv")},
                    oracle.pairwise(z), TOL[prec])
    other = np.ascontiguousarray(masks[::-1])
    P2 = h.plv_analytic_bands(xt, torch.tensor(other))
    P3 = h.plv_analytic_bands(xt, torch.tensor(masks))
    torch.cuda.synchronize()
    assert torch.equal(P3, P)
    assert torch.equal(P2[0], P[len(BANDS) - 1])


def test_bands_rejections(handles):
    h = handles["bf16x3"]
    for T in (1, 12289, 16384):
        x = torch.zeros((1, 4, T), device="cuda")
        with pytest.raises(PlvError):
            h.plv_analytic_bands(x, torch.zeros((2, T // 2 + 1)))
    # lengths outside the power-of-two kernel read the masks back: refused
    # inside a stream capture (and nothing is captured)
    T = 1000
    x = torch.zeros((1, 4, T), device="cuda")
    m = torch.ones((1, T // 2 + 1), device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(PlvError):
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                h.plv_analytic_bands(x, m)
    torch.cuda.synchronize()
