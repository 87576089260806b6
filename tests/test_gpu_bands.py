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


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("B,N,T", [(1, 7, 128), (2, 33, 1024), (1, 130, 4096), (1, 3, 8192)])
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
    for b in range(len(BANDS)):
        got = unpack_phasors(P[b].view(torch.float32), prec, B, N, T)
        z = oracle.analytic_band(xf, masks[b].astype(np.float64))
        a = np.abs(z)
        ref = np.where(a > 0, z / np.where(a > 0, a, 1), 0)
        rms = np.sqrt(np.mean(a ** 2))
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


def test_bands_rejections(handles):
    h = handles["bf16x3"]
    for T in (1000, 64, 16384):
        x = torch.zeros((1, 4, T), device="cuda")
        with pytest.raises(PlvError):
            h.plv_analytic_bands(x, torch.zeros((2, T // 2 + 1)))
