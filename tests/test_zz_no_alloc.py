"""plv_backward_noalloc: the backward pass for callers that cannot allocate
device memory (it runs on a fixed static scratch array instead of handle
scratch).  Called through the C ABI, its output must match plv_backward's on
two calls in a row (different inputs, so stale scratch would show).

This file is collected last on purpose: when it fails, a run that stops at
the first failure has already run every other test.  It passes alone in a
fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest
import torch


pytestmark = pytest.mark.gpu


def test_noalloc_backward_matches_allocating_backward():
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import _lib, synth
    h = plv.Handle(precision="fp32")
    lib = h.lib
    B, N, T = 2, 96, 1024  # well inside the fixed scratch array
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        x = synth.bandlimited(B, N, T, seed=77 + call, device="cuda")
        P = h.plv_analytic(x)
        C = h.plv_gram(P, B, N, T, plv=False, iplv=False, ciplv=False,
                       C=True)["C"]
        g = torch.Generator(device="cuda").manual_seed(5 + call)
        g1 = torch.randn(B, N, N, device="cuda", generator=g)
        g3 = torch.randn(B, N, N, device="cuda", generator=g)
        ref = h.plv_backward(x, C, g1, None, g3)
        out = torch.full_like(ref, float("nan"))
        rc = lib.plv_backward_noalloc(stream, ctypes.c_void_p(x.data_ptr()),
                                      _lib.PLV_F32, B, N, T, T,
                                      ctypes.c_void_p(C.data_ptr()),
                                      ctypes.c_void_p(g1.data_ptr()), None,
                                      ctypes.c_void_p(g3.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()))
        assert rc == _lib.PLV_OK, lib.plv_last_error(None)
        torch.cuda.synchronize()
        # the FP32 handle's backward runs the same kernels on the same values
        assert torch.equal(out, ref), call
        if call == 0:
            # and it is the gradient: FP64 autograd through plain torch ops
            from oracle import backward as obw
            e = 1
            want = obw.torch_grad(x[e].double().cpu().numpy(), g1[e].double().cpu().numpy(),
                                  None, g3[e].double().cpu().numpy())
            got = out[e].double().cpu().numpy()
            rel2 = np.linalg.norm(got - want) / np.linalg.norm(want)
            err = np.abs(got - want).max() / np.abs(want).max()
            assert rel2 < 5e-4 and err < 2e-3, (rel2, err)
    h.close()


def test_noalloc_backward_rejects_oversized_problem():
    import paper_1710_08037_gb300 as plv  # noqa: F401
    from paper_1710_08037_gb300 import _lib
    lib = _lib.load()
    rc = lib.plv_backward_noalloc(None, None, _lib.PLV_F32, 16, 1024, 4096,
                                  4096, None, None, None, None,
                                  ctypes.c_void_p(16))
    assert rc == _lib.PLV_ERR_INVALID
    assert b"scratch" in lib.plv_last_error(None)
