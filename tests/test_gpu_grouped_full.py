"""The uneven-batch workload at full size, in the launch configuration the
benchmark times: 256 subjects x 5 bands (1280 problems, N 68..2000,
T 500..10000), one autotuned plan, the grouped analytic signal and the
grouped Gram each replayed from a CUDA graph.  Sampled pairs of several
problems (the extremes of N and T among them) against the FP64 oracle, and
invariants on every output."""
import numpy as np
import pytest
import torch

import oracle
from bench import grouped_problems
from paper_1710_08037_gb300 import synth
from tests.helpers import DIAG_TOL, TOL, compare

pytestmark = pytest.mark.gpu


def test_full_grouped_workload_sampled():
    import paper_1710_08037_gb300 as plv
    torch.cuda.empty_cache()
    prec = "bf16x3"
    h = plv.Handle(precision=prec)
    specs = grouped_problems(seed=1004, nsub=256)
    probs = []
    for (N, T, band, sd) in specs:
        x = synth.bandlimited(1, N, T, seed=sd, band=band, device="cuda")
        h.prepare(T)
        probs.append({"x": x, "P": h.empty_phasors(1, N, T), "batch": 1,
                      "N": N, "T": T})
    grp = h.plv_group_create(probs, diag=True)
    h.plv_analytic_grouped(grp)
    h.plv_gram_grouped(grp)
    torch.cuda.synchronize()
    h.plv_group_tune(grp, reps=1)
    s = torch.cuda.Stream()
    g1, g2 = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g1, stream=s):
            h.plv_analytic_grouped(grp)
        with torch.cuda.graph(g2, stream=s):
            h.plv_gram_grouped(grp)
    for q in probs:
        q["plv"].fill_(float("nan"))
    g1.replay()
    g2.replay()
    torch.cuda.synchronize()
    assert h.plv_sync_status() == 0

    Ns = np.array([q["N"] for q in probs])
    Ts = np.array([q["T"] for q in probs])
    rng = np.random.default_rng(1004)
    pick = {int(np.argmax(Ns)), int(np.argmin(Ns)), int(np.argmax(Ts)),
            int(np.argmin(Ts))} | set(int(v) for v in rng.choice(len(probs), 3,
                                                                 replace=False))
    worst = {"plv": 0.0, "iplv": 0.0, "ciplv": 0.0}
    for p in sorted(pick):
        q = probs[p]
        N = q["N"]
        rows = rng.choice(N, size=min(4, N), replace=False)
        cols = rng.choice(N, size=min(16, N), replace=False)
        pi, pj = np.repeat(rows, len(cols)), np.tile(cols, len(rows))
        ref = oracle.connectivity_pairs(q["x"][0].double().cpu().numpy(), pi, pj)
        ii, jj = torch.tensor(pi, device="cuda"), torch.tensor(pj, device="cuda")
        gpu = {k: q[k][0][ii, jj].double().cpu().numpy()
               for k in ("plv", "iplv", "ciplv")}
        errs = compare(gpu, ref, TOL[prec])
        for k in worst:
            worst[k] = max(worst[k], errs[k])
    print("grouped full-size worst errors over problems", sorted(pick), worst)
    # invariants on every problem's whole output
    for q in probs:
        assert float(q["diag"].max()) < DIAG_TOL[prec], (q["N"], q["T"])
        assert not bool(torch.isnan(q["plv"]).any()), (q["N"], q["T"])
        assert float(q["plv"].max()) <= 1.0 + 1e-5
        assert bool(torch.all(q["iplv"] <= q["plv"] + 1e-6))
        assert torch.equal(q["plv"][0], q["plv"][0].T)
        assert torch.equal(q["ciplv"][0], -q["ciplv"][0].T)
    grp.close()
    h.close()
    del probs
    torch.cuda.empty_cache()
