"""Shared helpers for the GPU parity tests: reading the phasor operand
layout back, and the tolerance rules."""
import numpy as np
import torch

# Gram arithmetic tolerances against the FP64 oracle (absolute, on C, PLV and
# iPLV).  FP32 path: 1e-5.  BF16x3 path: BF16 keeps 8 significant bits, so
# hi = RN(p) is within 2^-8 |p| and hi + lo within 2^-16 |p|; with the dropped
# lo*lo term (<= 2^-16 |p q|) every product term of the Gram carries at most
# 3 * 2^-16 ~ 4.6e-5 |p q| (worst case, all errors aligned).  The mean over T
# samples averages these rounding errors; the stated bound, 2e-5, is an
# empirical margin (about 2x the largest error measured against the oracle
# at full size, 9.1e-6 on the diagonal at N = T = 8192, where the tensor
# core's truncating accumulation over 1024-sample chunks adds to it).  FP16x3 (11 significant bits): 3 * 2^-22 ~ 7e-7 per
# term, stated 1e-5.
TOL = {"fp32": 1e-5, "bf16x3": 2e-5, "fp16x3": 1e-5}
# phasor (operand) representation tolerance and diagonal |C_ii - 1| bound
PHASOR_TOL = {"fp32": 2e-6, "bf16x3": 4e-5, "fp16x3": 3e-6}
DIAG_TOL = {"fp32": 1e-6, "bf16x3": 3e-5, "fp16x3": 2e-6}


def unpack_phasors(P, precision, B, N, T):
    """Operand buffer -> complex128 numpy (B, N, T) (layout of plv.h)."""
    ld = ((T + 31) // 32) * 32
    if precision == "fp32":
        a = P[: B * N * 2 * ld].view(B, N, 2, ld).double().cpu().numpy()
        return a[:, :, 0, :T] + 1j * a[:, :, 1, :T]
    # tiled split layout: blocks [B][NRB][NKB][4 planes][128 rows][32], the
    # 16-byte chunk c of row r stored at chunk c ^ ((r >> 1) & 3)
    dt = torch.bfloat16 if precision == "bf16x3" else torch.float16
    nrb, nkb = (N + 127) // 128, ld // 32
    b = P.view(dt)[: B * nrb * nkb * 4 * 128 * 32].double().cpu().numpy()
    b = b.reshape(B, nrb, nkb, 4, 128, 4, 8)
    r = np.arange(128)
    chunk = np.arange(4)
    src = chunk[None, :] ^ ((r[:, None] >> 1) & 3)          # (128, 4)
    b = b[:, :, :, :, r[:, None], src, :]                   # unswizzle
    b = b.transpose(0, 3, 1, 4, 2, 5, 6).reshape(B, 4, nrb * 128, ld)
    b = b[:, :, :N, :T]
    return (b[:, 0] + b[:, 1]) + 1j * (b[:, 2] + b[:, 3])


def ciplv_bound(c, eps):
    """First-order error bound of ciPLV given an absolute error eps on Re C
    and Im C: eps/sqrt(d) + |Im Re| eps / d^(3/2), d = 1 - Re^2 (Eq. 14)."""
    re, im = c.real, c.imag
    d = np.maximum((1 - re) * (1 + re), 1e-12)
    return eps / np.sqrt(d) + np.abs(im * re) * eps / d ** 1.5


def compare(gpu, ref, eps, off_diag_only=False):
    """Assert |gpu - ref| within eps for PLV / iPLV and the conditioned
    bound for ciPLV; ref holds the oracle's c, plv, iplv, ciplv (numpy)."""
    c = ref["c"]
    errs = {}
    for k in ("plv", "iplv"):
        e = np.abs(gpu[k] - ref[k])
        errs[k] = float(e.max()) if e.size else 0.0
        assert errs[k] <= eps, (k, errs[k])
    bound = ciplv_bound(c, eps) + 1e-6
    e = np.abs(gpu["ciplv"] - ref["ciplv"])
    bad = e > bound
    if off_diag_only:
        pass
    assert not np.any(bad), ("ciplv", float(e.max()), int(bad.sum()))
    errs["ciplv"] = float(e.max()) if e.size else 0.0
    return errs
