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
