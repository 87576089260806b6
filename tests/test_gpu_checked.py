"""The bounds-checked build (PLV_CHECKED, libplv_checked.so): small odd
shapes through the whole path, the grouped plan and the backward pass,
against the FP64 oracle, with no out-of-range access caught by the kernels'
bounds conditions (plv_check_status reports 0)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1710_08037_gb300 import synth
from tests.helpers import TOL, compare

pytestmark = pytest.mark.gpu

SHAPES = [(1, 500), (3, 997), (67, 1000), (129, 500), (3, 32), (67, 128), (129, 4096),
          (200, 997)]


@pytest.fixture(scope="module", params=["fp32", "bf16x3", "fp16x3"])
def hc(request):
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision=request.param, checked=True)
    assert h.lib.plv_build_checked() == 1
    assert h.check_status() == 0
    yield h
    h.close()


def _np(res):
    return {k: v.double().cpu().numpy() for k, v in res.items() if k in ("plv", "iplv", "ciplv")}


@pytest.mark.parametrize("N,T", SHAPES)
def test_checked_path_small_odd_shapes(hc, N, T):
    prec = {0: "fp32", 1: "bf16x3", 2: "fp16x3"}[hc.precision]
    x = synth.bandlimited(2, N, T, seed=N * 7 + T, band=(5.0, 40.0), device="cuda")
    res = _np(hc.connectivity(x))
    assert hc.check_status() == 0
    for e in range(2):
        ref = oracle.connectivity(x[e].double().cpu().numpy())
        compare({k: v[e] for k, v in res.items()}, ref, TOL[prec])


def test_checked_grouped_and_windows(hc):
    prec = {0: "fp32", 1: "bf16x3", 2: "fp16x3"}[hc.precision]
    probs, xs = [], []
    for N, T in SHAPES[:5]:
        x = synth.bandlimited(1, N, T, seed=N + T, device="cuda")
        hc.prepare(T)
        xs.append(x)
        probs.append({"x": x, "P": hc.empty_phasors(1, N, T), "batch": 1, "N": N, "T": T})
    if hc.precision != 0:
        grp = hc.plv_group_create(probs)
        hc.plv_analytic_grouped(grp)
        hc.plv_gram_grouped(grp)
        torch.cuda.synchronize()
        assert hc.check_status() == 0
        for q, x in zip(grp.problems, xs):
            ref = oracle.connectivity(x[0].double().cpu().numpy())
            compare({k: q[k][0].double().cpu().numpy() for k in ("plv", "iplv", "ciplv")}, ref,
                    TOL[prec])
        grp.close()
    # sliding windows of 96 samples at a hop of 64 over T = 1000
    N, T = 67, 1000
    x = synth.bandlimited(1, N, T, seed=99, device="cuda")
    P = hc.plv_analytic(x)
    nw = (T - 96) // 64 + 1
    res = hc.plv_gram_windows(P, 1, N, T, 0, 96, 64, nw)
    torch.cuda.synchronize()
    assert hc.check_status() == 0
    assert torch.isfinite(res["plv"]).all()


def test_checked_backward(hc):
    rng = np.random.default_rng(3)
    N, T = 67, 500
    x = synth.bandlimited(2, N, T, seed=5, device="cuda")
    C = hc.plv_gram(hc.plv_analytic(x), 2, N, T, C=True)["C"]
    g = torch.tensor(rng.standard_normal((2, N, N)), device="cuda", dtype=torch.float32)
    grad = hc.plv_backward(x, C, None, None, g)
    torch.cuda.synchronize()
    assert hc.check_status() == 0
    assert torch.isfinite(grad).all()


def test_checked_split_k(hc):
    """Split-K parts (long tiles of a grouped plan) under the bounds checks."""
    if hc.precision == 0:
        pytest.skip("split K is a tensor-core Gram schedule")
    prec = {1: "bf16x3", 2: "fp16x3"}[hc.precision]
    probs, xs = [], []
    for N, T in ((68, 10000), (130, 4096), (3, 7000)):
        x = synth.bandlimited(1, N, T, seed=N + 3 * T, device="cuda")
        hc.prepare(T)
        xs.append(x)
        probs.append({"x": x, "P": hc.empty_phasors(1, N, T), "batch": 1, "N": N, "T": T})
    grp = hc.plv_group_create(probs)
    hc.plv_group_configure(grp, gram_split=4)
    hc.plv_analytic_grouped(grp)
    hc.plv_gram_grouped(grp)
    torch.cuda.synchronize()
    assert hc.check_status() == 0
    for q, x in zip(grp.problems, xs):
        ref = oracle.connectivity(x[0].double().cpu().numpy())
        compare({k: q[k][0].double().cpu().numpy() for k in ("plv", "iplv", "ciplv")}, ref,
                TOL[prec])
    grp.close()
