"""Sliding-window Grams through the C ABI (plv_gram_windows) against the
oracle's pairwise definition on each window's samples, for every operand
precision; one whole-length window equals plv_gram bit for bit."""
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


def _check(res, ref, prec, b):
    for w in range(ref["c"].shape[0]):
        gpu = {k: res[k][b, w].double().cpu().numpy() for k in ("plv", "iplv", "ciplv")}
        compare(gpu, {k: ref[k][w] for k in ("c", "plv", "iplv", "ciplv")}, TOL[prec])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,T,t0,W,hop,nw", [(70, 300, 32, 64, 32, 7), (130, 256, 0, 128, 64, 3),
                                             (9, 96, 64, 32, 0, 2)])
def test_windows_on_given_phasors(handles, prec, N, T, t0, W, hop, nw):
    """Eq. 4 on a random complex signal, then the windowed Gram, against the
    pairwise definition on each window (ragged N, T not a multiple of 32)."""
    h = handles[prec]
    rng = np.random.default_rng(N + T)
    B = 2
    z = rng.standard_normal((B, N, T)) + 1j * rng.standard_normal((B, N, T))
    P = h.plv_normalize(torch.tensor(z, device="cuda", dtype=torch.complex64))
    res = h.plv_gram_windows(P, B, N, T, t0, W, hop, nw, diag=True)
    torch.cuda.synchronize()
    for b in range(B):
        zb = z[b].astype(np.complex64).astype(np.complex128)
        _check(res, oracle.windows(zb, t0, W, hop, nw), prec, b)
    assert float(res["diag"].max()) < 1e-4


@pytest.mark.parametrize("prec", PRECS)
def test_windows_from_signals(handles, prec):
    """x -> analytic signal -> windows, against the oracle's analytic signal
    of the whole epoch and the pairwise definition per window."""
    h = handles[prec]
    E, N, T = 2, 40, 1024
    x = synth.bandlimited(E, N, T, seed=88, band=(8, 30), device="cuda")
    P = h.plv_analytic(x)
    res = h.plv_gram_windows(P, E, N, T, 64, 256, 128, 6)
    torch.cuda.synchronize()
    for b in range(E):
        z = oracle.analytic(x[b].double().cpu().numpy())
        _check(res, oracle.windows(z, 64, 256, 128, 6), prec, b)


@pytest.mark.parametrize("prec", PRECS)
def test_single_window_equals_plv_gram(handles, prec):
    h = handles[prec]
    E, N, T = 3, 100, 512
    x = synth.bandlimited(E, N, T, seed=5, device="cuda")
    P = h.plv_analytic(x)
    a = h.plv_gram(P, E, N, T)
    b = h.plv_gram_windows(P, E, N, T, 0, T, 0, 1)
    torch.cuda.synchronize()
    for k in ("plv", "iplv", "ciplv"):
        assert torch.equal(a[k], b[k][:, 0]), k


def test_windows_rejections(handles):
    h = handles["bf16x3"]
    P = h.empty_phasors(1, 8, 100)
    with pytest.raises(PlvError):
        h.plv_gram_windows(P, 1, 8, 100, 0, 48, 32, 2)    # W not a multiple of 32
    with pytest.raises(PlvError):
        h.plv_gram_windows(P, 1, 8, 100, 32, 64, 32, 2)   # second window ends past T
