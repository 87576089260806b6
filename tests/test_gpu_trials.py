"""Grams over trials through the C ABI: the time-resolved PLV (Eq. 1 / 8)
and coherency across trials (Eq. 12), against the FP64 oracle over trials,
with ragged trial counts, rows and columns, zero samples and zero channels."""
import numpy as np
import pytest
import torch

import oracle
from paper_1710_08037_gb300 import PlvError, synth
from tests.helpers import TOL, compare

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "bf16x3", "fp16x3"]


@pytest.fixture(scope="module")
def handles():
    import paper_1710_08037_gb300 as plv
    hs = {p: plv.Handle(precision=p) for p in PRECS}
    yield hs
    for h in hs.values():
        h.close()


def _planar(z):
    """complex (E, N, L) -> FP32 planar rows (E, N, 2, ld) on the device."""
    E, N, L = z.shape
    ld = (L + 31) // 32 * 32
    V = np.zeros((E, N, 2, ld), np.float32)
    V[:, :, 0, :L] = z.real
    V[:, :, 1, :L] = z.imag
    return torch.tensor(V, device="cuda"), ld


def _check(res, ref, prec, keys=("plv", "iplv", "ciplv")):
    for l in range(ref["c"].shape[0]):
        gpu = {k: res[k][l].double().cpu().numpy() for k in ("plv", "iplv", "ciplv")}
        r = {"c": ref["c"][l]}
        for k, rk in zip(("plv", "iplv", "ciplv"), keys):
            r[k] = ref[rk][l]
        compare(gpu, r, TOL[prec])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("E,N,T,l0,L", [(20, 37, 100, 10, 50), (33, 129, 64, 0, 64),
                                        (64, 8, 40, 5, 33), (1, 3, 32, 0, 32)])
def test_time_resolved_gram_vs_oracle(handles, prec, E, N, T, l0, L):
    """Unit phasors of the oracle's analytic signal through plv_trial_operands
    (mode asis) and plv_gram against Eq. 1 evaluated with phases; one sample
    is zero (it contributes nothing, the normaliser stays 1/E)."""
    h = handles[prec]
    rng = np.random.default_rng(E * 1000 + N + T)
    z = oracle.analytic(rng.standard_normal((E, N, T)))
    z[0, min(1, N - 1), l0 + 2] = 0.0
    a = np.abs(z)
    p = np.where(a > 0, z / np.where(a > 0, a, 1.0), 0.0)
    V, ld = _planar(p)
    P = h.plv_trial_operands(V, E, N, ld, l0, L, "asis")
    res = h.plv_gram(P, L, N, E)
    torch.cuda.synchronize()
    _check(res, oracle.time_resolved(z, l0, L), prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("T", [64, 96])
def test_time_resolved_end_to_end_tones(handles, prec, T):
    """x -> analytic signal (K1) -> trial operands -> Gram on on-bin tones
    with a common phase per trial: PLV(t) = 1, iPLV(t) = |sin(delta_i -
    delta_j)|, ciPLV(t) = its sign, against the oracle over trials."""
    h = handles[prec]
    rng = np.random.default_rng(T)
    E, N, k = 24, 10, 5
    theta = rng.uniform(0, 2 * np.pi, E)
    delta = rng.uniform(0, 2 * np.pi, N)
    t = np.arange(T)
    x = np.cos(2 * np.pi * k * t[None, None] / T + theta[:, None, None]
               + delta[None, :, None])
    res = h.time_resolved(torch.tensor(x, device="cuda", dtype=torch.float32), 3, T - 6)
    torch.cuda.synchronize()
    ref = oracle.time_resolved(oracle.analytic(x.astype(np.float32).astype(np.float64)),
                               3, T - 6)
    _check(res, ref, prec)
    assert float((res["plv"] - 1).abs().max()) < 1e-4


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("E,N,T,f0,F", [(30, 20, 256, 8, 12), (7, 131, 100, 0, 40)])
def test_coherency_vs_oracle(handles, prec, E, N, T, f0, F):
    """Fourier coefficients at selected bins (the oracle's direct DFT)
    through mode rms and plv_gram: coherence, imaginary coherency and lagged
    coherence of Eq. 12 against the oracle; one channel is zero."""
    h = handles[prec]
    x = synth.bandlimited(E, N, T, seed=E + N, band=(5, 120)).double().numpy()
    x[:, 4] = 0.0
    X = oracle.dft_bins(x, f0, F)
    ref = oracle.coherency_trials(X)
    res = h.coherency(torch.tensor(X, device="cuda", dtype=torch.complex64))
    torch.cuda.synchronize()
    _check(res, ref, prec, keys=("coh", "icoh", "lcoh"))
    assert float(res["plv"][:, 4].abs().max()) == 0.0


def test_trial_operands_rejections(handles):
    h = handles["bf16x3"]
    V = torch.zeros((2, 3, 2, 32), device="cuda")
    with pytest.raises(PlvError):
        h.plv_trial_operands(V, 2, 3, 32, 10, 30, "asis")   # l0 + L > ldv
    with pytest.raises(PlvError):
        h.plv_trial_operands(V, 0, 3, 32, 0, 8, "asis")     # no trials
    from paper_1710_08037_gb300 import _lib
    P = h.empty_phasors(8, 3, 2)
    rc = h.lib.plv_trial_operands(h.h, None, V.data_ptr(), 2, 3, 32, 0, 8, 7, P.data_ptr())
    assert rc == _lib.PLV_ERR_INVALID                        # unknown mode


@pytest.mark.parametrize("T,f0,F", [(256, 3, 20), (1000, 40, 70), (4096, 0, 33), (97, 1, 96)])
def test_dft_bins_vs_oracle(handles, T, f0, F):
    """The device DFT at selected bins against the oracle's FP64 direct sum
    (F > 32 splits over launches; odd and prime T)."""
    h = handles["fp32"]
    rows = 300
    x = synth.bandlimited(1, rows, T, seed=T + F, band=(5, 200))[0].double().numpy()
    X = h.plv_dft_bins(torch.tensor(x, device="cuda", dtype=torch.float32), f0, F)
    torch.cuda.synchronize()
    got = (X[:, 0, :F] + 1j * X[:, 1, :F]).cpu().numpy().astype(np.complex128)
    ref = oracle.dft_bins(x.astype(np.float32).astype(np.float64), f0, F)
    rms = np.sqrt(np.mean(x ** 2))
    err = np.abs(got - ref)
    assert err.max() < 1e-5 * np.sqrt(T) * rms, err.max() / (np.sqrt(T) * rms)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 3e-6


@pytest.mark.parametrize("prec", PRECS)
def test_coherency_from_signals_vs_oracle(handles, prec):
    """x -> DFT at bins -> trial operands (RMS) -> Gram, all on the device,
    against the oracle's direct DFT and coherency across trials."""
    h = handles[prec]
    E, N, T, f0, F = 40, 45, 512, 4, 24
    x = synth.bandlimited(E, N, T, seed=77, band=(4, 60)).numpy()
    res = h.coherency_bins(torch.tensor(x, device="cuda"), f0, F)
    torch.cuda.synchronize()
    X = oracle.dft_bins(x.astype(np.float64), f0, F)
    _check(res, oracle.coherency_trials(X), prec, keys=("coh", "icoh", "lcoh"))
