"""Gradient references for the differentiable PLV / iPLV / ciPLV path.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Two independent references for dL/dx, L = sum_ij (g_plv PLV + g_iplv iPLV +
g_ciplv ciPLV)_ij, with x the real input signals:

* ``fd_grad``: FP64 central finite differences of the C oracle's forward
  (direct-DFT analytic signal, Eq. 3; pairwise definition, Eq. 2; read-outs,
  Eq. 7, 13, 14).  Entirely independent of any analytic derivative.
* ``torch_grad``: a plain FP64 PyTorch-CPU graph of the reformulated path
  (library FFT -> analytic mask -> inverse FFT -> z/|z| (Eq. 4) ->
  P P^H / T (Eq. 7) -> read-outs) differentiated by autograd.

The two pin each other: they share no arithmetic.
"""
from __future__ import annotations

import numpy as np
import torch

from . import connectivity


def loss_value(x: np.ndarray, g_plv, g_iplv, g_ciplv) -> float:
    """L(x) for one epoch x (N, T), evaluated with the FP64 oracle."""
    out = connectivity(x)
    L = 0.0
    if g_plv is not None:
        L += float(np.sum(g_plv * out["plv"]))
    if g_iplv is not None:
        L += float(np.sum(g_iplv * out["iplv"]))
    if g_ciplv is not None:
        L += float(np.sum(g_ciplv * out["ciplv"]))
    return L


def fd_grad(x: np.ndarray, g_plv=None, g_iplv=None, g_ciplv=None,
            entries=None, rel_step: float = 1e-6) -> np.ndarray:
    """Central finite differences of ``loss_value`` at the flat indices
    ``entries`` of x (default: all).  Step h = rel_step * max(1, |x|)."""
    x = np.array(x, dtype=np.float64)
    flat = x.reshape(-1)
    if entries is None:
        entries = np.arange(flat.size)
    g = np.empty(len(entries))
    for k, q in enumerate(entries):
        h = rel_step * max(1.0, abs(flat[q]))
        old = flat[q]
        flat[q] = old + h
        lp = loss_value(x, g_plv, g_iplv, g_ciplv)
        flat[q] = old - h
        lm = loss_value(x, g_plv, g_iplv, g_ciplv)
        flat[q] = old
        g[k] = (lp - lm) / (2.0 * h)
    return g


def _hmask(T: int) -> torch.Tensor:
    h = torch.zeros(T, dtype=torch.float64)
    h[0] = 1.0
    if T % 2 == 0:
        h[1:T // 2] = 2.0
        h[T // 2] = 1.0
    else:
        h[1:(T + 1) // 2] = 2.0
    return h


def torch_forward(x: torch.Tensor):
    """Plain-torch FP64 forward of the reformulated path for x (..., N, T).
    Returns (C, plv, iplv, ciplv)."""
    T = x.shape[-1]
    z = torch.fft.ifft(torch.fft.fft(x.to(torch.complex128), dim=-1)
                       * _hmask(T), dim=-1)
    a = z.abs()
    P = torch.where(a > 0, z / torch.where(a > 0, a, torch.ones_like(a)),
                    torch.zeros_like(z))
    C = P @ P.mH / T
    R, I = C.real, C.imag
    plv = C.abs()
    iplv = I.abs()
    d = (1.0 - R) * (1.0 + R)
    ok = d > 0
    ciplv = torch.where(ok, I / torch.sqrt(torch.where(ok, d,
                                                       torch.ones_like(d))),
                        torch.zeros_like(d))
    eye = torch.eye(x.shape[-2], dtype=torch.bool)
    iplv = torch.where(eye, torch.zeros_like(iplv), iplv)
    ciplv = torch.where(eye, torch.zeros_like(ciplv), ciplv)
    return C, plv, iplv, ciplv


def torch_grad(x: np.ndarray, g_plv=None, g_iplv=None, g_ciplv=None):
    """dL/dx by FP64 autograd through ``torch_forward``."""
    xt = torch.tensor(np.asarray(x, dtype=np.float64), requires_grad=True)
    _, plv, iplv, ciplv = torch_forward(xt)
    L = torch.zeros((), dtype=torch.float64)
    if g_plv is not None:
        L = L + (torch.as_tensor(g_plv, dtype=torch.float64) * plv).sum()
    if g_iplv is not None:
        L = L + (torch.as_tensor(g_iplv, dtype=torch.float64) * iplv).sum()
    if g_ciplv is not None:
        L = L + (torch.as_tensor(g_ciplv, dtype=torch.float64) * ciplv).sum()
    L.backward()
    return xt.grad.numpy()
