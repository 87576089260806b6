"""Autotuner of grouped plans through the C ABI: every launch shape it can
choose (thread class per transform length, CTAs per SM, Gram tile schedule)
gives the same phasors and the same outputs as the plan's default shape;
split K, which regroups a split tile's FP32 additions, gives the same
phasors, outputs within FP32 rounding of the unsplit plan's, and the same
bits on every run.  The tuned plan reproduces its results, the choice is
cached per work signature, and CUDA graphs captured before tuning keep
working."""
import numpy as np
import pytest
import torch

import oracle
from paper_1710_08037_gb300 import synth
from tests.helpers import TOL, ciplv_bound, compare

pytestmark = pytest.mark.gpu

# (batch, N, T): transform lengths M in all four thread classes (768, 1280,
# 2048, 4096, 10240, 20480), a power-of-two T, a single row, and enough Gram tiles
# (> 152) that the balanced schedule differs from longest first
SHAPES = [(1, 70, 600), (2, 1600, 1000), (1, 200, 2000), (1, 130, 5000),
          (1, 40, 9000), (1, 256, 1024), (1, 1, 333)]
KEYS = ("plv", "iplv", "ciplv", "C", "diag")


def _plan(h, seed0=500):
    probs = []
    for k, (B, N, T) in enumerate(SHAPES):
        x = synth.bandlimited(B, N, T, seed=seed0 + k, device="cuda")
        probs.append({"x": x, "P": h.empty_phasors(B, N, T), "batch": B,
                      "N": N, "T": T})
    grp = h.plv_group_create(probs, C=True, diag=True)
    return probs, grp


def _phasor_values(P, prec):
    """Operand bytes as numbers (a zero's sign aside, equal values are
    equal bits)."""
    if prec == "fp32":
        return P.view(torch.float32).clone()
    return P.view(torch.bfloat16 if prec == "bf16x3" else torch.float16).float()


def _run(h, grp, probs):
    """Zero the phasors (padding rows stay zero) and poison the outputs, then
    run the plan: a tile or row pair the launches skip shows up."""
    for q in probs:
        q["P"].zero_()
        for k in ("plv", "iplv", "ciplv"):
            q[k].fill_(float("nan"))
        q["C"].fill_(complex(float("nan"), 0.0))
        q["diag"].fill_(float("nan"))
    h.plv_analytic_grouped(grp)
    h.plv_gram_grouped(grp)
    torch.cuda.synchronize()
    assert h.plv_sync_status() == 0


def _snapshot(probs, prec):
    return [({k: q[k].clone() for k in KEYS}, _phasor_values(q["P"], prec))
            for q in probs]


def _assert_same(ref, probs, prec, what):
    for (outs, P), q in zip(ref, probs):
        assert torch.equal(P, _phasor_values(q["P"], prec)), (what, q["N"], q["T"], "P")
        for k in KEYS:
            assert torch.equal(outs[k], q[k]), (what, q["N"], q["T"], k)


# split K against the unsplit plan: the part sums and their sum regroup the
# FP32 additions of a tile's chunk sums (a few per tile, each of magnitude
# <= T): a few FP32 roundings of C, about 1e-7, allowed 1e-6
SPLIT_EPS = 1e-6


def _assert_close(ref, probs, prec, what):
    for (outs, P), q in zip(ref, probs):
        assert torch.equal(P, _phasor_values(q["P"], prec)), (what, q["N"], q["T"], "P")
        c = outs["C"].cpu().numpy().astype(np.complex128)
        for k in ("plv", "iplv", "diag"):
            e = float((outs[k].double() - q[k].double()).abs().max())
            assert e <= SPLIT_EPS, (what, q["N"], q["T"], k, e)
        e = float((outs["C"] - q["C"]).abs().max())
        assert e <= SPLIT_EPS, (what, q["N"], q["T"], "C", e)
        eb = np.abs(outs["ciplv"].double().cpu().numpy() - q["ciplv"].double().cpu().numpy())
        assert np.all(eb <= ciplv_bound(c, SPLIT_EPS) + 1e-7), (what, q["N"], q["T"], "ciplv")


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_every_candidate_shape_gives_the_same_results(prec):
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision=prec)
    probs, grp = _plan(h)
    _run(h, grp, probs)
    ref = _snapshot(probs, prec)
    # the default shape agrees with the oracle (row 0 of the smaller problems)
    for q in probs:
        if q["N"] <= 256:
            want = oracle.connectivity(q["x"][0].double().cpu().numpy())
            got = {k: q[k][0].double().cpu().numpy() for k in ("plv", "iplv", "ciplv")}
            compare(got, want, TOL[prec])
    configs = [dict(k1_widen=True),
               dict(k1_per_sm=[1, 1, 1, 1]),
               dict(k1_widen=True, k1_per_sm=[2, 2, 1, 1]),
               dict(gram_schedule="balanced_rounds", gram_tile_cost=0),
               dict(gram_schedule="balanced_rounds", gram_tile_cost=32)]
    for cfg in configs:
        h.plv_group_configure(grp, **cfg)
        _run(h, grp, probs)
        _assert_same(ref, probs, prec, cfg)
    # split K of the 9000- and 5000-sample tiles (diagonal tiles among them)
    for cfg in (dict(gram_split=1),
                dict(gram_split=4, gram_schedule="balanced_rounds", gram_tile_cost=8)):
        h.plv_group_configure(grp, **cfg)
        _run(h, grp, probs)
        (_assert_same if prec == "fp32" else _assert_close)(ref, probs, prec, cfg)
        again = _snapshot(probs, prec)
        _run(h, grp, probs)
        _assert_same(again, probs, prec, ("split K, second run", cfg))
    grp.close()
    h.close()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
def test_tuned_plan_reproduces_default_results_and_is_cached(prec):
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision=prec)
    probs, grp = _plan(h)
    _run(h, grp, probs)
    ref = _snapshot(probs, prec)
    # a graph captured before tuning keeps the lists it was captured with
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            h.plv_analytic_grouped(grp)
            h.plv_gram_grouped(grp)
    torch.cuda.synchronize()
    r = h.plv_group_tune(grp, reps=2)
    assert r["cached"] == 0 and r["timed_configs"] > 0
    assert r["k1_lengths"] == 6  # M = 20480, 10240, 4096, 2048, 1280, 768
    assert 1 <= r["k1_launches"] <= 4
    assert 0 <= r["k1_widened"] <= r["k1_lengths"]
    assert r["k1_ms_default"] > 0 and 0 < r["k1_ms_tuned"] <= r["k1_ms_default"]
    assert r["gram_ms_default"] > 0 and 0 < r["gram_ms_tuned"] <= r["gram_ms_default"]
    _run(h, grp, probs)
    (_assert_close if r["gram_split"] else _assert_same)(ref, probs, prec, "tuned")
    for q in probs:
        q["P"].zero_()
        q["plv"].fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    _assert_same(ref, probs, prec, "graph captured before tuning")
    # tuning the same plan again, or an equal plan, applies the cached choice
    r2 = h.plv_group_tune(grp, reps=2)
    assert r2["cached"] == 1 and r2["timed_configs"] == 0
    for k in ("k1_widened", "k1_per_sm", "gram_schedule", "gram_tile_cost", "gram_split",
              "gram_split_tiles"):
        assert r2[k] == r[k], k
    probs2, grp2 = _plan(h, seed0=900)
    r3 = h.plv_group_tune(grp2, reps=2)
    assert r3["cached"] == 1 and r3["gram_schedule"] == r["gram_schedule"]
    grp2.close()
    grp.close()
    h.close()


def test_tuner_rejects_bad_arguments():
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300._lib import PlvError
    h = plv.Handle(precision="bf16x3")
    probs, grp = _plan(h)
    with pytest.raises(PlvError):
        h.plv_group_tune(grp, reps=0)
    with pytest.raises(PlvError):
        h.plv_group_configure(grp, k1_per_sm=[-1, 0, 0, 0])
    with pytest.raises(PlvError):
        h.plv_group_configure(grp, gram_tile_cost=-5)
    with pytest.raises(PlvError):
        h.plv_group_configure(grp, gram_split=65)
    other = plv.Handle(precision="fp16x3")
    with pytest.raises(PlvError):
        other.plv_group_tune(grp)
    other.close()
    grp.close()
    h.close()


# few long tiles: a plan that leaves most of the grid idle without split K
LONG = [(1, 68, 10000), (2, 100, 8000), (1, 250, 9999), (1, 129, 4096)]


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
def test_split_k_results_in_graphs_and_after_tuning(prec):
    """Split K: each part stores its sums and the last part of a block adds
    them in part order.  Every split factor agrees with the oracle and with
    the unsplit plan to FP32 rounding, gives the same bits on every run and
    from a CUDA graph (the counters' memset is part of the graph), and so
    does the factor the tuner keeps."""
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision=prec)
    probs = []
    for k, (B, N, T) in enumerate(LONG):
        x = synth.bandlimited(B, N, T, seed=700 + k, device="cuda")
        probs.append({"x": x, "P": h.empty_phasors(B, N, T), "batch": B, "N": N, "T": T})
    grp = h.plv_group_create(probs, C=True, diag=True)
    # the host plan splits every tile of this plan at f = 1
    chunk = 32 if prec == "bf16x3" else 4
    nkb = []
    for B, N, T in LONG:
        nrb = (N + 127) // 128
        nkb += [plv.phasor_ld(T) // 32] * (B * nrb * (nrb + 1) // 2)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert min(plv.gram_split_plan(nkb, chunk, sms, 1)) >= 2
    _run(h, grp, probs)
    ref = _snapshot(probs, prec)
    wants = [oracle.connectivity(q["x"][0].double().cpu().numpy()) for q in probs[:2]]
    for f in (1, 2, 4, 64):
        h.plv_group_configure(grp, gram_split=f)
        _run(h, grp, probs)
        _assert_close(ref, probs, prec, ("split", f))
        for q, want in zip(probs, wants):
            got = {k: q[k][0].double().cpu().numpy() for k in ("plv", "iplv", "ciplv")}
            compare(got, want, TOL[prec])
        first = _snapshot(probs, prec)
        _run(h, grp, probs)  # the counters start from zero in every launch
        _assert_same(first, probs, prec, ("split again", f))
    # a graph of the split plan, replayed twice
    h.plv_group_configure(grp, gram_split=2)
    _run(h, grp, probs)
    ref = _snapshot(probs, prec)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            h.plv_analytic_grouped(grp)
            h.plv_gram_grouped(grp)
    torch.cuda.synchronize()
    for rep in range(2):
        for q in probs:
            q["P"].zero_()
            for k in ("plv", "iplv", "ciplv"):
                q[k].fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        assert h.plv_sync_status() == 0
        _assert_same(ref, probs, prec, ("graph replay", rep))
    # the tuner: whatever it keeps agrees with the unsplit plan
    h.plv_group_configure(grp)
    _run(h, grp, probs)
    ref = _snapshot(probs, prec)
    r = h.plv_group_tune(grp, reps=2)
    assert r["gram_split"] in (0, 1, 2, 4)
    assert (r["gram_split_tiles"] > 0) == (r["gram_split"] > 0)
    _run(h, grp, probs)
    _assert_close(ref, probs, prec, ("tuned", r["gram_split"]))
    grp.close()
    h.close()
