"""Grouped Gram (one persistent launch over problems of uneven N and T)
through the C ABI: each problem's outputs equal the single-problem launch
bit for bit and the oracle within tolerance; the whole group replays
identically from a CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
from paper_1710_08037_gb300 import synth
from tests.helpers import TOL, compare

pytestmark = pytest.mark.gpu

SHAPES = [(2, 68, 256), (1, 130, 1024), (3, 257, 512), (1, 1000, 4096),
          (2, 5, 64), (1, 128, 2048)]


def _problems(h):
    probs = []
    for k, (B, N, T) in enumerate(SHAPES):
        x = synth.bandlimited(B, N, T, seed=300 + k, device="cuda")
        probs.append({"x": x, "P": h.plv_analytic(x), "batch": B, "N": N,
                      "T": T})
    return probs


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3", "fp32"])
def test_grouped_equals_single_and_oracle(prec):
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision=prec)
    probs = _problems(h)
    grp = h.plv_group_create(probs, C=True, diag=True)
    h.plv_gram_grouped(grp)
    torch.cuda.synchronize()
    assert h.plv_sync_status() == 0
    for q in probs:
        single = h.plv_gram(q["P"], q["batch"], q["N"], q["T"], C=True,
                            diag=True)
        for k in ("plv", "iplv", "ciplv", "C"):
            assert torch.equal(single[k], q[k]), (q["N"], q["T"], k)
        if q["N"] <= 257:
            e = q["batch"] - 1
            ref = oracle.connectivity(q["x"][e].double().cpu().numpy())
            gpu = {k: q[k][e].double().cpu().numpy()
                   for k in ("plv", "iplv", "ciplv")}
            compare(gpu, ref, TOL[prec])
    grp.close()
    h.close()


def test_grouped_in_cuda_graph():
    """Capture the phasor kernels of every problem and the grouped Gram in
    one CUDA graph; replays give identical results."""
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision="bf16x3")
    probs = _problems(h)
    grp = h.plv_group_create(probs)
    h.plv_gram_grouped(grp)  # warm-up outside capture
    torch.cuda.synchronize()
    first = {k: [q[k].clone() for q in probs] for k in ("plv", "ciplv")}
    for q in probs:
        q["plv"].zero_()
        q["ciplv"].zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            for q in probs:
                h.plv_analytic(q["x"], q["P"])
            h.plv_gram_grouped(grp)
    for _ in range(2):
        for q in probs:
            q["plv"].zero_()
        g.replay()
        torch.cuda.synchronize()
        for k in ("plv", "ciplv"):
            for a, q in zip(first[k], probs):
                assert torch.equal(a, q[k])
    grp.close()
    h.close()


# uneven lengths across the four thread classes of the any-length engine
# (M = 64 .. 24576), odd and power-of-two T, N off the 128-row tiles
K1_SHAPES = [(1, 70, 500), (2, 33, 1000), (1, 129, 2500), (1, 40, 4096),
             (1, 17, 5000), (1, 12, 9999), (3, 9, 33), (1, 200, 777),
             (1, 6, 12288), (2, 1, 100)]


def _k1_problems(h, dtype=torch.float32, poison=True):
    probs = []
    for k, (B, N, T) in enumerate(K1_SHAPES):
        x = synth.bandlimited(B, N, T, seed=400 + k, device="cuda").to(dtype)
        P = h.empty_phasors(B, N, T)
        if poison:  # everything the plan and the kernel must overwrite
            P.view(torch.uint8).fill_(0xFF)
        probs.append({"x": x, "P": P, "batch": B, "N": N, "T": T})
    return probs


def _pow2(T):
    return T & (T - 1) == 0


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3", "fp32"])
def test_grouped_analytic_equals_single(prec):
    """plv_analytic_grouped writes, for every problem, the same phasor bytes
    as plv_analytic (the same engine and plan) for lengths that are not a
    power of two, and agrees within the phasor tolerance where plv_analytic
    takes the direct power-of-two engine."""
    import paper_1710_08037_gb300 as plv
    from tests.helpers import PHASOR_TOL, unpack_phasors
    h = plv.Handle(precision=prec)
    probs = _k1_problems(h)
    grp = h.plv_group_create(probs)
    h.plv_analytic_grouped(grp)
    torch.cuda.synchronize()
    assert h.plv_sync_status() == 0
    for q in probs:
        B, N, T = q["batch"], q["N"], q["T"]
        single = h.empty_phasors(B, N, T)
        h.plv_analytic(q["x"], single)
        torch.cuda.synchronize()
        if not _pow2(T):
            assert torch.equal(single.view(torch.uint8), q["P"].view(torch.uint8)), (N, T)
        else:
            # two FFT algorithms: compare in z (a phasor's error is the
            # transform's error in z over |z|)
            a = unpack_phasors(single, prec, B, N, T)
            b = unpack_phasors(q["P"], prec, B, N, T)
            z = oracle.analytic(q["x"].double().cpu().numpy())
            rms = np.sqrt(np.mean(np.abs(z) ** 2))
            err_z = np.abs(a - b) * np.abs(z)
            assert err_z.max() < 2 * max(1e-5, PHASOR_TOL[prec]) * rms, (N, T)
    grp.close()
    h.close()


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_grouped_analytic_and_gram_vs_oracle(prec):
    """The whole grouped path (phasors and Gram of every problem from two
    calls on one plan) against the FP64 oracle on each problem's last
    epoch; the split layout's padding rows were poisoned before planning."""
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision=prec)
    probs = _k1_problems(h)
    grp = h.plv_group_create(probs, diag=True)
    h.plv_analytic_grouped(grp)
    h.plv_gram_grouped(grp)
    torch.cuda.synchronize()
    assert h.plv_sync_status() == 0
    for q in probs:
        e = q["batch"] - 1
        ref = oracle.connectivity(q["x"][e].double().cpu().numpy())
        gpu = {k: q[k][e].double().cpu().numpy()
               for k in ("plv", "iplv", "ciplv")}
        compare(gpu, ref, TOL[prec])
        assert float(q["diag"].max()) < 1e-4
    grp.close()
    h.close()


def test_grouped_analytic_f64_input_and_graph():
    """FP64 inputs through the grouped engine, captured with the grouped
    Gram in one CUDA graph: replays reproduce the eager outputs."""
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision="bf16x3")
    probs = _k1_problems(h, dtype=torch.float64)
    grp = h.plv_group_create(probs)
    h.plv_analytic_grouped(grp)
    h.plv_gram_grouped(grp)
    torch.cuda.synchronize()
    first = [q["ciplv"].clone() for q in probs]
    for q in probs[:3]:
        e = q["batch"] - 1
        ref = oracle.connectivity(q["x"][e].cpu().numpy())
        compare({k: q[k][e].double().cpu().numpy()
                 for k in ("plv", "iplv", "ciplv")}, ref, TOL["bf16x3"])
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            h.plv_analytic_grouped(grp)
            h.plv_gram_grouped(grp)
    for _ in range(2):
        for q in probs:
            q["ciplv"].zero_()
            q["P"].zero_()
        g.replay()
        torch.cuda.synchronize()
        for a, q in zip(first, probs):
            assert torch.equal(a, q["ciplv"])
    grp.close()
    h.close()


def test_grouped_analytic_rejections():
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import PlvError
    h = plv.Handle(precision="bf16x3")
    probs = _k1_problems(h, poison=False)[:2]
    probs[1]["x"] = probs[1]["x"].double()
    with pytest.raises(PlvError):  # two input dtypes in one plan
        h.plv_group_create(probs)
    no_x = [{k: v for k, v in q.items() if k != "x"} for q in probs]
    grp = h.plv_group_create(no_x)
    with pytest.raises(PlvError):  # a plan without inputs
        h.plv_analytic_grouped(grp)
    grp.close()
    x = torch.zeros((1, 4, 20000), device="cuda")
    big = [{"x": x, "P": h.empty_phasors(1, 4, 20000), "batch": 1, "N": 4,
            "T": 20000}]
    with pytest.raises(PlvError):  # longer than the engine's largest length
        h.plv_group_create(big)
    h.close()
