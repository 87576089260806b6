"""GPU parity of the backward pass (through the C ABI): against FP64
autograd through plain torch ops and against FP64 central finite
differences of the C oracle."""
import numpy as np
import pytest
import torch

from oracle import backward as obw
from paper_1710_08037_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h32():
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision="fp32")
    yield h
    h.close()


# the contraction Gamma = S P / T runs on the CUDA cores (FP32 handle) or on
# the tensor cores in BF16 hi + lo splits (split handles)
@pytest.fixture(scope="module", params=["fp32", "bf16x3"])
def hb(request):
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision=request.param)
    yield h
    h.close()


def _grads(rng, B, N, which):
    out = []
    for w in ("plv", "iplv", "ciplv"):
        if w in which:
            g = rng.standard_normal((B, N, N))
            out.append(g)
        else:
            out.append(None)
    return out


def _gpu_grad(h, x, gs):
    hf = h
    xd = torch.tensor(x, device="cuda", dtype=torch.float32)
    E, N, T = x.shape
    P = hf.plv_analytic(xd)
    C = hf.plv_gram(P, E, N, T, plv=False, iplv=False, ciplv=False, C=True)["C"]
    gt = [None if g is None else torch.tensor(g, device="cuda",
                                              dtype=torch.float32) for g in gs]
    g = h.plv_backward(xd, C, *gt)
    torch.cuda.synchronize()
    return g.double().cpu().numpy()


@pytest.mark.parametrize("which", [("plv",), ("iplv",), ("ciplv",),
                                   ("plv", "iplv", "ciplv")])
@pytest.mark.parametrize("N,T", [(16, 256), (67, 128), (20, 300)])
def test_backward_vs_torch_fp64(hb, which, N, T):
    rng = np.random.default_rng(N * 7 + T + len(which))
    B = 2
    x = synth.bandlimited(B, N, T, seed=N + T, fs=1000.0, band=(8, 60),
                          dtype=torch.float64).numpy()
    x = x.astype(np.float32).astype(np.float64)
    gs = _grads(rng, B, N, which)
    got = _gpu_grad(hb, x, gs)
    ref = np.stack([obw.torch_grad(x[e], *(None if g is None else g[e]
                                           for g in gs)) for e in range(B)])
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max() / scale
    rel2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 2e-3 and rel2 < 5e-4, (err, rel2)


def test_backward_vs_finite_differences(hb):
    """FP64 central differences of the oracle's forward (direct DFT + the
    pairwise loop) at 24 entries, N = 16, T = 256."""
    rng = np.random.default_rng(5)
    N, T = 16, 256
    x = rng.standard_normal((1, N, T)).astype(np.float32).astype(np.float64)
    g1 = rng.standard_normal((N, N))
    g3 = rng.standard_normal((N, N))
    np.fill_diagonal(g3, 0.0)
    got = _gpu_grad(hb, x, [g1[None], None, g3[None]])[0].reshape(-1)
    ent = rng.choice(N * T, size=24, replace=False)
    fd = obw.fd_grad(x[0], g1, None, g3, entries=ent)
    scale = np.abs(got).max()
    assert np.max(np.abs(got[ent] - fd)) < 1e-3 * scale


def test_ciplv_loss_workload_sampled(hb):
    """The differentiable-loss workload: 16 recordings, N = 1024, T = 4096,
    loss = sum of ciPLV over a seeded 10 % pair mask; two recordings checked
    against FP64 autograd through plain torch ops."""
    B, N, T = 16, 1024, 4096
    x = synth.bandlimited(B, N, T, seed=1005, device="cuda")
    mask = synth.random_pair_mask(N, 0.10, seed=1005, device="cuda")
    g3 = mask.to(torch.float32).expand(B, N, N).contiguous()
    P = hb.plv_analytic(x)
    C = hb.plv_gram(P, B, N, T, plv=False, iplv=False, ciplv=False,
                    C=True)["C"]
    g = hb.plv_backward(x, C, None, None, g3)
    torch.cuda.synchronize()
    assert torch.isfinite(g).all()
    for e in (0, 11):
        xe = x[e].double().cpu().numpy()
        ref = obw.torch_grad(xe, None, None, mask.double().cpu().numpy())
        got = g[e].double().cpu().numpy()
        rel2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        print("ciPLV loss backward: rel2", rel2, "max rel", err)
        assert rel2 < 1e-3 and err < 5e-3


def test_autograd_function(hb):
    """connectivity() is a torch.autograd.Function whose backward is
    plv_backward; its gradient matches FP64 autograd of plain torch ops."""
    import paper_1710_08037_gb300 as plv
    rng = np.random.default_rng(9)
    N, T = 12, 128
    x = rng.standard_normal((1, N, T)).astype(np.float32)
    xd = torch.tensor(x, device="cuda", requires_grad=True)
    p, ip, cp = plv.connectivity(xd, hb)
    w = torch.tensor(rng.standard_normal((1, N, N)), device="cuda",
                     dtype=torch.float32)
    (p * w).sum().add((cp * w.transpose(1, 2)).sum()).backward()
    ref = obw.torch_grad(x[0].astype(np.float64), w[0].double().cpu().numpy(),
                         None, w[0].T.double().cpu().numpy())
    got = xd.grad[0].double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 5e-4


def test_backward_zero_grads_and_validation(h32):
    from paper_1710_08037_gb300 import _lib
    x = torch.randn(1, 8, 64, device="cuda")
    C = torch.zeros(1, 8, 8, dtype=torch.complex64, device="cuda")
    g = h32.plv_backward(x, C)
    assert torch.all(g == 0)
    xl = torch.randn(1, 8, 20000, device="cuda")
    rc = h32.lib.plv_backward(h32.h, None, xl.data_ptr(), 0, 1, 8, 20000, 20000,
                              C.data_ptr(), C.data_ptr(), None, None, g.data_ptr())
    assert rc == _lib.PLV_ERR_UNSUPPORTED


@pytest.mark.parametrize("N,T", [(67, 300), (130, 1000), (200, 129), (33, 4096)])
def test_tensor_core_contraction_equals_fp32(h32, N, T):
    """The split-precision backward (S and conj(P)^T as BF16 split rows, the
    contraction on the tensor cores) against the FP32 CUDA-core backward on
    the same x and C, at sizes that leave ragged 32- and 128-blocks in both
    operands."""
    import paper_1710_08037_gb300 as plv
    rng = np.random.default_rng(N + T)
    B = 3
    x = synth.bandlimited(B, N, T, seed=N * T, band=(8, 60), device="cuda")
    P = h32.plv_analytic(x)
    C = h32.plv_gram(P, B, N, T, plv=False, iplv=False, ciplv=False, C=True)["C"]
    gs = [torch.tensor(rng.standard_normal((B, N, N)), device="cuda",
                       dtype=torch.float32) for _ in range(3)]
    ref = h32.plv_backward(x, C, *gs)
    hs = plv.Handle(precision="bf16x3")
    got = hs.plv_backward(x, C, *gs)
    torch.cuda.synchronize()
    assert hs.plv_sync_status() == 0
    rel = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
    err = float((got - ref).abs().max() / ref.abs().max())
    assert rel < 2e-5 and err < 1e-4, (rel, err)
    hs.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_graph_keeps_its_scratch_after_growth(prec):
    """A CUDA graph captured with plv_backward keeps the scratch it was
    captured with: a later, larger eager call grows the handle's scratch,
    and replaying the older graph still gives the eager gradient bit for
    bit (the buffer it used is kept until the handle is destroyed)."""
    import paper_1710_08037_gb300 as plv
    h = plv.Handle(precision=prec)
    rng = np.random.default_rng(21)
    B, N, T = 2, 96, 256
    x = synth.bandlimited(B, N, T, seed=31, device="cuda")
    C = h.plv_gram(h.plv_analytic(x), B, N, T, plv=False, iplv=False, ciplv=False,
                   C=True)["C"]
    g3 = torch.tensor(rng.standard_normal((B, N, N)), device="cuda", dtype=torch.float32)
    want = h.plv_backward(x, C, None, None, g3)  # sizes the scratch outside capture
    grad = torch.empty_like(want)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            h.plv_backward(x, C, None, None, g3, grad_x=grad)
    # a larger problem grows the scratch (eagerly)
    B2, N2, T2 = 3, 300, 1024
    x2 = synth.bandlimited(B2, N2, T2, seed=32, device="cuda")
    C2 = h.plv_gram(h.plv_analytic(x2), B2, N2, T2, plv=False, iplv=False, ciplv=False,
                    C=True)["C"]
    g32 = torch.tensor(rng.standard_normal((B2, N2, N2)), device="cuda", dtype=torch.float32)
    h.plv_backward(x2, C2, None, None, g32)
    grad.zero_()
    with torch.cuda.stream(s):
        graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(grad, want)
    assert h.plv_sync_status() == 0
    del graph
    h.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("N,T", [(67, 300), (130, 1024), (33, 4096), (129, 1000)])
def test_saved_backward_equals_recompute(prec, N, T):
    """plv_backward_saved on plv_analytic_save's outputs gives plv_backward's
    gradient bit for bit (same x, same C): the saved phasors are the
    recompute's.  The saved forward's Gram agrees with the FP64 oracle."""
    import oracle
    import paper_1710_08037_gb300 as plv
    from tests.helpers import TOL, compare
    h = plv.Handle(precision=prec)
    B = 2
    x = synth.bandlimited(B, N, T, seed=N + 7 * T, band=(8, 60), device="cuda")
    saved = h.plv_analytic_save(x)
    res = h.plv_gram(saved["P"], B, N, T, C=True)
    C = res["C"]
    rng = np.random.default_rng(N * T)
    gs = [torch.tensor(rng.standard_normal((B, N, N)), device="cuda", dtype=torch.float32)
          for _ in range(3)]
    a = h.plv_backward(x, C, *gs)
    b = h.plv_backward_saved(saved, C, *gs)
    c = h.plv_backward_saved(saved, C, None, None, gs[2])
    d = h.plv_backward(x, C, None, None, gs[2])
    torch.cuda.synchronize()
    assert h.plv_sync_status() == 0
    assert torch.equal(a, b)
    assert torch.equal(c, d)
    ref = oracle.connectivity(x[0].double().cpu().numpy())
    compare({k: res[k][0].double().cpu().numpy() for k in ("plv", "iplv", "ciplv")}, ref,
            TOL[prec])
    h.close()


def test_saved_mode_autograd():
    """connectivity(recompute=False) keeps the phasors for the backward pass:
    its gradient of a ciPLV loss matches the recomputing path's (their
    forward phasors differ only in the last bits on a BF16X3 handle), and
    FP16X3 handles refuse the saved form."""
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import _lib
    h = plv.Handle(precision="bf16x3")
    B, N, T = 2, 96, 2048
    x0 = synth.bandlimited(B, N, T, seed=31, band=(8, 40), device="cuda")
    rng = np.random.default_rng(5)
    w = torch.tensor(rng.standard_normal((B, N, N)), device="cuda", dtype=torch.float32)
    grads = []
    for recompute in (True, False):
        x = x0.clone().requires_grad_(True)
        _, _, ciplv = plv.connectivity(x, h, recompute=recompute)
        (ciplv * w).sum().backward()
        grads.append(x.grad.detach().clone())
    rel = float(torch.linalg.norm(grads[0] - grads[1]) / torch.linalg.norm(grads[0]))
    assert rel < 1e-4, rel
    h16 = plv.Handle(precision="fp16x3")
    with pytest.raises(_lib.PlvError) as ei:
        h16.plv_analytic_save(x0)
    assert ei.value.status == _lib.PLV_ERR_UNSUPPORTED
    h16.close()
    h.close()
