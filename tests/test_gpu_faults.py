"""Failure detection on the GPU without a GPU fault: host-side injected
allocation and launch failures (plv_debug_fault) return their status codes
and leave the handle usable, and the tensor-core Gram's bounded pipeline
wait, made to run out by a withheld operand copy under a short bound
(plv_set_wait_limit), ends the launch with PLV_ERR_TIMEOUT in the device
status word while the context stays usable for the next, correct call."""
import numpy as np
import pytest
import torch

import oracle
from paper_1710_08037_gb300 import _lib, synth
from tests.helpers import TOL, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def disarm():
    import paper_1710_08037_gb300 as plv  # noqa: F401  (loads the library)
    lib = _lib.load()
    lib.plv_debug_fault(_lib.PLV_FAULT_NONE, 0)
    yield lib
    lib.plv_debug_fault(_lib.PLV_FAULT_NONE, 0)


def _armed(lib):
    return lib.plv_debug_fault_armed(None)


@pytest.mark.parametrize("countdown", [1, 2])
def test_allocation_failure_in_create(disarm, countdown):
    """plv_create's first or second device allocation fails: PLV_ERR_ALLOC,
    nothing is handed out, and the next create works."""
    import paper_1710_08037_gb300 as plv
    lib = disarm
    assert lib.plv_debug_fault(_lib.PLV_FAULT_ALLOC, countdown) == _lib.PLV_OK
    with pytest.raises(plv.PlvError) as ei:
        plv.Handle(precision="bf16x3")
    assert ei.value.status == _lib.PLV_ERR_ALLOC
    assert _armed(lib) == _lib.PLV_FAULT_NONE
    h = plv.Handle(precision="bf16x3")
    assert h.plv_sync_status() == 0
    h.close()


def test_allocation_failure_in_plan_and_scratch(disarm):
    """The any-length plan (plv_prepare) and the backward scratch fail to
    allocate once each; the calls report PLV_ERR_ALLOC and succeed when
    repeated, with the same results as a handle that never failed."""
    import paper_1710_08037_gb300 as plv
    lib = disarm
    h = plv.Handle(precision="fp32")
    ref = plv.Handle(precision="fp32")
    lib.plv_debug_fault(_lib.PLV_FAULT_ALLOC, 1)
    with pytest.raises(plv.PlvError) as ei:
        h.prepare(1000)
    assert ei.value.status == _lib.PLV_ERR_ALLOC
    h.prepare(1000)
    x = synth.bandlimited(1, 20, 1000, seed=3, device="cuda")
    assert torch.equal(h.plv_analytic(x), ref.plv_analytic(x))
    C = ref.plv_gram(ref.plv_analytic(x), 1, 20, 1000, C=True)["C"]
    g = torch.randn(1, 20, 20, device="cuda")
    lib.plv_debug_fault(_lib.PLV_FAULT_ALLOC, 1)
    with pytest.raises(plv.PlvError) as ei:
        h.plv_backward(x, C, g)
    assert ei.value.status == _lib.PLV_ERR_ALLOC
    assert torch.equal(h.plv_backward(x, C, g), ref.plv_backward(x, C, g))
    h.close()
    ref.close()


def test_allocation_failure_in_group_create(disarm):
    import paper_1710_08037_gb300 as plv
    lib = disarm
    h = plv.Handle(precision="bf16x3")
    probs = []
    for N, T in ((70, 500), (130, 256)):
        x = synth.bandlimited(1, N, T, seed=N, device="cuda")
        h.prepare(T)
        probs.append({"x": x, "P": h.empty_phasors(1, N, T), "batch": 1, "N": N, "T": T})
    lib.plv_debug_fault(_lib.PLV_FAULT_ALLOC, 1)
    with pytest.raises(plv.PlvError) as ei:
        h.plv_group_create(probs)
    assert ei.value.status == _lib.PLV_ERR_ALLOC
    grp = h.plv_group_create(probs)
    h.plv_analytic_grouped(grp)
    h.plv_gram_grouped(grp)
    torch.cuda.synchronize()
    assert h.plv_sync_status() == 0
    grp.close()
    h.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_launch_failure_launches_nothing(disarm, prec):
    """An injected launch failure of plv_gram returns PLV_ERR_CUDA without
    launching: the outputs keep their poison; the next call is correct."""
    import paper_1710_08037_gb300 as plv
    lib = disarm
    h = plv.Handle(precision=prec)
    x, _ = synth.tones(seed=1001)
    xd = torch.tensor(x, device="cuda")
    P = h.plv_analytic(xd)
    N, T = x.shape[1], x.shape[2]
    out = {k: torch.full((1, N, N), float("nan"), device="cuda") for k in ("plv", "iplv", "ciplv")}
    lib.plv_debug_fault(_lib.PLV_FAULT_LAUNCH, 1)
    with pytest.raises(plv.PlvError) as ei:
        h.plv_gram(P, 1, N, T, out=out)
    assert ei.value.status == _lib.PLV_ERR_CUDA
    torch.cuda.synchronize()
    assert all(bool(torch.isnan(v).all()) for v in out.values())
    res = h.plv_gram(P, 1, N, T, out=out)
    ref = oracle.connectivity(x[0])
    compare({k: res[k][0].double().cpu().numpy() for k in ("plv", "iplv", "ciplv")}, ref,
            TOL[prec])
    assert h.plv_sync_status() == 0
    h.close()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
def test_bounded_wait_times_out_and_the_context_survives(disarm, prec):
    """Every CTA of one Gram launch withholds its first operand copy, so its
    MMA issuer's wait for that stage never completes and runs into a 20 ms
    bound: plv_sync_status reports PLV_ERR_TIMEOUT.  With the default bound
    restored, the next launch on the same handle matches the oracle and
    leaves the status clean."""
    import paper_1710_08037_gb300 as plv
    lib = disarm
    h = plv.Handle(precision=prec)
    x, _ = synth.tones(seed=1001)
    xd = torch.tensor(x, device="cuda")
    N, T = x.shape[1], x.shape[2]
    P = h.plv_analytic(xd)
    h.set_wait_limit(20_000_000)
    lib.plv_debug_fault(_lib.PLV_FAULT_STALL, 1)
    h.plv_gram(P, 1, N, T)
    assert _armed(lib) == _lib.PLV_FAULT_NONE
    assert h.plv_sync_status() == _lib.PLV_ERR_TIMEOUT
    assert h.plv_sync_status() == 0  # read and cleared
    h.set_wait_limit(0)
    res = h.plv_gram(P, 1, N, T)
    ref = oracle.connectivity(x[0])
    compare({k: res[k][0].double().cpu().numpy() for k in ("plv", "iplv", "ciplv")}, ref,
            TOL[prec])
    assert h.plv_sync_status() == 0
    # a larger problem after the timeout: all tiles, several chunks per tile
    xb = synth.bandlimited(2, 600, 2048, seed=44, device="cuda")
    other = plv.Handle(precision=prec)
    a = h.connectivity(xb)
    b = other.connectivity(xb)
    for k in ("plv", "iplv", "ciplv"):
        assert torch.equal(a[k], b[k]), k
    assert h.plv_sync_status() == 0
    other.close()
    h.close()


def test_short_bound_without_a_stall_changes_nothing(disarm):
    """A 20 ms bound is far above any normal pipeline wait: a clean launch
    under it gives the default bound's bits and no timeout."""
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision="bf16x3")
    x = synth.bandlimited(2, 700, 4096, seed=45, device="cuda")
    P = h.plv_analytic(x)
    a = h.plv_gram(P, 2, 700, 4096)
    h.set_wait_limit(20_000_000)
    b = h.plv_gram(P, 2, 700, 4096)
    for k in ("plv", "iplv", "ciplv"):
        assert torch.equal(a[k], b[k]), k
    assert h.plv_sync_status() == 0
    h.close()
    assert np.isfinite(float(a["plv"].max()))


def test_memory_high_water_mark(disarm):
    """plv_memory_usage: the handle's own device bytes (tables, plans,
    scratch) now and at most; a new plan and the backward scratch raise
    both."""
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision="fp32")
    cur0, peak0 = h.memory_usage()
    assert cur0 > 0 and peak0 == cur0
    h.prepare(1000)
    cur1, peak1 = h.memory_usage()
    assert cur1 > cur0 and peak1 == cur1
    x = synth.bandlimited(1, 40, 1000, seed=8, device="cuda")
    C = h.plv_gram(h.plv_analytic(x), 1, 40, 1000, C=True)["C"]
    g = torch.randn(1, 40, 40, device="cuda")
    h.plv_backward(x, C, g)
    cur2, peak2 = h.memory_usage()
    ld = 1024
    assert cur2 >= cur1 + 40 * ld * 20 and peak2 == cur2
    h.close()
