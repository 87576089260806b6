"""GB300 Phase Locking Value: Python binding of the C ABI (include/plv.h).

    import torch, paper_1710_08037_gb300 as plv
    h = plv.Handle(precision="bf16x3")
    out = h.connectivity(x)           # x: (E, N, T) float32 / float64, cuda
    out["plv"], out["iplv"], out["ciplv"]   # (E, N, N) float32 each

The functions mirror the C entry points (``plv_analytic``, ``plv_gram``, ...)
and only marshal arguments: torch supplies device memory and the current
stream; every computation runs in the library's CUDA kernels.  There is no
CPU fallback -- without a GPU or without the built library, calls raise.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import (PLV_F32, PLV_F64, PLV_OUT_C, PLV_OUT_CIPLV, PLV_OUT_IPLV,
                   PLV_OUT_PLV, PLV_PREC_BF16X3, PLV_PREC_FP16X3,
                   PLV_PREC_FP32, PlvError)

__all__ = ["Handle", "PlvError", "phasor_ld", "connectivity",
           "PLV_PREC_FP32", "PLV_PREC_BF16X3", "PLV_PREC_FP16X3"]

_PREC = {"fp32": PLV_PREC_FP32, "bf16x3": PLV_PREC_BF16X3,
         "fp16x3": PLV_PREC_FP16X3, PLV_PREC_FP32: PLV_PREC_FP32,
         PLV_PREC_BF16X3: PLV_PREC_BF16X3, PLV_PREC_FP16X3: PLV_PREC_FP16X3}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dtype_code(t):
    if t.dtype in (torch.float32, torch.complex64):
        return PLV_F32
    if t.dtype in (torch.float64, torch.complex128):
        return PLV_F64
    raise PlvError(_lib.PLV_ERR_INVALID, f"unsupported dtype {t.dtype}")


def phasor_ld(T: int) -> int:
    """Padded row length of the phasor operand layout."""
    return int(_lib.load().plv_phasor_ld(int(T)))


class Handle:
    """Owns a ``plv_handle`` (device, Gram precision, workspace)."""

    def __init__(self, precision="fp32", device=None, workspace_limit=0, checked=False):
        """checked=True runs on the bounds-checked build of the library
        (libplv_checked.so, PLV_CHECKED): see check_status()."""
        if not torch.cuda.is_available():
            raise PlvError(_lib.PLV_ERR_UNSUPPORTED,
                           "no CUDA device: this library has no CPU path")
        self.lib = _lib.load(checked=checked)
        self.checked = bool(checked)
        self.device = torch.device("cuda", torch.cuda.current_device()
                                   if device is None else int(device))
        self.precision = _PREC[precision]
        h = ctypes.c_void_p()
        _lib.check(self.lib.plv_create(ctypes.byref(h), self.device.index,
                                       self.precision, int(workspace_limit)), None, self.lib)
        self.h = h
        if checked:
            _lib._checked_handles.add(h.value)

    def close(self):
        if getattr(self, "_h32", None) is not None:
            self._h32.close()
            self._h32 = None
        if getattr(self, "h", None):
            _lib._checked_handles.discard(self.h.value)
            self.lib.plv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- C entry points ---------------------------------------------------
    def phasor_bytes(self, batch, N, T) -> int:
        return int(self.lib.plv_phasor_bytes(self.h, batch, N, T))

    def empty_phasors(self, batch, N, T):
        nb = self.phasor_bytes(batch, N, T)
        return torch.empty(max(nb, 16) // 4, dtype=torch.float32,
                           device=self.device)

    def prepare(self, T: int):
        _lib.check(self.lib.plv_prepare(self.h, int(T)), self.h)

    def plv_analytic(self, x, P=None):
        """Eq. 3 + 4: x (batch, N, T) real on the device -> phasors P."""
        assert x.is_cuda and x.dim() == 3
        B, N, T = x.shape
        if not (x.stride(-1) == 1 and (N == 1 or x.stride(0) == N * x.stride(1))):
            x = x.contiguous()
        ldx = x.stride(1) if N > 1 else max(x.stride(0), T)
        if P is None:
            P = self.empty_phasors(B, N, T)
        _lib.check(self.lib.plv_analytic(self.h, _stream(self.device), _ptr(x),
                                         _dtype_code(x), B, N, T, ldx,
                                         _ptr(P)), self.h)
        return P

    def plv_analytic_bands(self, x, masks, P=None):
        """Band-pass and Eq. 3 + 4 for every band of ``masks`` (nbands,
        T//2 + 1) float32 on the device: returns the phasors of the bands,
        (nbands, bytes of one buffer) uint8 (buffer b is P[b]).  Powers of
        two from 128 to 8192 take one forward FFT per row pair; any other T
        up to 12288 the any-length engine, which reads the masks back
        (synchronising the stream; not inside a graph capture)."""
        assert x.is_cuda and x.dim() == 3
        B, N, T = x.shape
        if not (x.stride(-1) == 1 and (N == 1 or x.stride(0) == N * x.stride(1))):
            x = x.contiguous()
        ldx = x.stride(1) if N > 1 else max(x.stride(0), T)
        masks = masks.to(device=x.device, dtype=torch.float32).contiguous()
        nb = masks.shape[0]
        assert masks.shape == (nb, T // 2 + 1)
        nbytes = self.lib.plv_phasor_bytes(self.h, B, N, T)
        if P is None:
            P = torch.empty((nb, nbytes), dtype=torch.uint8, device=x.device)
        _lib.check(self.lib.plv_analytic_bands(self.h, _stream(self.device), _ptr(x),
                                               _dtype_code(x), B, N, T, ldx, _ptr(masks),
                                               nb, _ptr(P)), self.h)
        return P

    def plv_normalize(self, z, P=None):
        """Eq. 4 on a given complex analytic signal z (batch, N, T)."""
        assert z.is_cuda and z.dim() == 3 and z.is_complex()
        z = z.contiguous()
        B, N, T = z.shape
        if P is None:
            P = self.empty_phasors(B, N, T)
        _lib.check(self.lib.plv_normalize(self.h, _stream(self.device),
                                          _ptr(z), _dtype_code(z), B, N, T, T,
                                          _ptr(P)), self.h)
        return P

    def plv_gram(self, P, batch, N, T, plv=True, iplv=True, ciplv=True,
                 C=False, diag=False, out=None):
        """Eq. 7, 13, 14: Gram of the phasors with fused read-outs."""
        dev = self.device
        res = {} if out is None else dict(out)

        def mk(key, want, shape, dtype):
            if not want:
                return None
            if key not in res:
                res[key] = torch.empty(shape, dtype=dtype, device=dev)
            return res[key]

        o_plv = mk("plv", plv, (batch, N, N), torch.float32)
        o_iplv = mk("iplv", iplv, (batch, N, N), torch.float32)
        o_ci = mk("ciplv", ciplv, (batch, N, N), torch.float32)
        o_C = mk("C", C, (batch, N, N), torch.complex64)
        o_d = mk("diag", diag, (batch,), torch.float64)
        mask = ((PLV_OUT_PLV if plv else 0) | (PLV_OUT_IPLV if iplv else 0) |
                (PLV_OUT_CIPLV if ciplv else 0) | (PLV_OUT_C if C else 0))
        _lib.check(self.lib.plv_gram(self.h, _stream(dev), _ptr(P), batch, N,
                                     T, mask, _ptr(o_plv), _ptr(o_iplv),
                                     _ptr(o_ci), _ptr(o_C), _ptr(o_d)),
                   self.h)
        return res

    def plv_gram_windows(self, P, batch, N, T, t0, W, hop, nw, plv=True, iplv=True,
                         ciplv=True, C=False, diag=False, out=None):
        """Sliding-window Grams (Eq. 7 over windows of W samples starting at
        t0 + w hop, w < nw) with the read-outs: dict of (batch, nw, N, N)."""
        dev = self.device
        res = {} if out is None else dict(out)

        def mk(key, want, shape, dtype):
            if not want:
                return None
            if key not in res:
                res[key] = torch.empty(shape, dtype=dtype, device=dev)
            return res[key]

        sh = (batch, nw, N, N)
        o_plv = mk("plv", plv, sh, torch.float32)
        o_iplv = mk("iplv", iplv, sh, torch.float32)
        o_ci = mk("ciplv", ciplv, sh, torch.float32)
        o_C = mk("C", C, sh, torch.complex64)
        o_d = mk("diag", diag, (batch, nw), torch.float64)
        mask = ((PLV_OUT_PLV if plv else 0) | (PLV_OUT_IPLV if iplv else 0) |
                (PLV_OUT_CIPLV if ciplv else 0) | (PLV_OUT_C if C else 0))
        _lib.check(self.lib.plv_gram_windows(self.h, _stream(dev), _ptr(P), batch, N, T,
                                             t0, W, hop, nw, mask, _ptr(o_plv),
                                             _ptr(o_iplv), _ptr(o_ci), _ptr(o_C),
                                             _ptr(o_d)), self.h)
        return res

    def plv_metrics(self, C):
        """Eq. 7, 13, 14 elementwise on a stored complex64 C (batch, N, N)."""
        assert C.is_cuda and C.dtype == torch.complex64
        C = C.contiguous()
        B, N, _ = C.shape
        res = {k: torch.empty((B, N, N), dtype=torch.float32,
                              device=self.device)
               for k in ("plv", "iplv", "ciplv")}
        _lib.check(self.lib.plv_metrics(self.h, _stream(self.device), _ptr(C),
                                        B, N, _ptr(res["plv"]),
                                        _ptr(res["iplv"]),
                                        _ptr(res["ciplv"])), self.h)
        return res

    def plv_backward(self, x, C, g_plv=None, g_iplv=None, g_ciplv=None,
                     grad_x=None):
        """Gradient of sum(g_plv PLV + g_iplv iPLV + g_ciplv ciPLV) with
        respect to x (batch, N, T); C is the forward's complex64 Gram."""
        assert x.is_cuda and x.dim() == 3 and C.dtype == torch.complex64
        B, N, T = x.shape
        if not (x.stride(-1) == 1 and (N == 1 or x.stride(0) == N * x.stride(1))):
            x = x.contiguous()
        ldx = x.stride(1) if N > 1 else max(x.stride(0), T)
        C = C.contiguous()
        gs = [None if g is None else g.to(torch.float32).contiguous()
              for g in (g_plv, g_iplv, g_ciplv)]
        if grad_x is None:
            grad_x = torch.empty((B, N, T), dtype=torch.float32,
                                 device=self.device)
        _lib.check(self.lib.plv_backward(self.h, _stream(self.device), _ptr(x),
                                         _dtype_code(x), B, N, T, ldx,
                                         _ptr(C), _ptr(gs[0]), _ptr(gs[1]),
                                         _ptr(gs[2]), _ptr(grad_x)), self.h)
        return grad_x

    def plv_analytic_save(self, x):
        """Eq. 3 + 4 in the form plv_backward_saved takes: returns a dict
        with the Gram operand "P" (for plv_gram), the FP32 planar phasors
        "P32" and "rinv" = 1/|z| [batch*N][ld].  FP32 and BF16X3 handles."""
        assert x.is_cuda and x.dim() == 3
        B, N, T = x.shape
        if not (x.stride(-1) == 1 and (N == 1 or x.stride(0) == N * x.stride(1))):
            x = x.contiguous()
        ldx = x.stride(1) if N > 1 else max(x.stride(0), T)
        ld = phasor_ld(T)
        P = self.empty_phasors(B, N, T)
        if self.precision == 0:
            P32 = P
        else:
            P32 = torch.empty(B * N * 2 * ld, dtype=torch.float32, device=self.device)
        rinv = torch.empty(B * N * ld, dtype=torch.float32, device=self.device)
        _lib.check(self.lib.plv_analytic_save(self.h, _stream(self.device), _ptr(x),
                                              _dtype_code(x), B, N, T, ldx, _ptr(P),
                                              _ptr(P32), _ptr(rinv)), self.h)
        return {"P": P, "P32": P32, "rinv": rinv, "shape": (B, N, T)}

    def plv_backward_saved(self, saved, C, g_plv=None, g_iplv=None, g_ciplv=None,
                           grad_x=None):
        """plv_backward from plv_analytic_save's outputs (no recompute)."""
        B, N, T = saved["shape"]
        assert C.dtype == torch.complex64
        C = C.contiguous()
        gs = [None if g is None else g.to(torch.float32).contiguous()
              for g in (g_plv, g_iplv, g_ciplv)]
        if grad_x is None:
            grad_x = torch.empty((B, N, T), dtype=torch.float32, device=self.device)
        _lib.check(self.lib.plv_backward_saved(self.h, _stream(self.device), B, N, T,
                                               _ptr(saved["P"]), _ptr(saved["P32"]),
                                               _ptr(saved["rinv"]), _ptr(C), _ptr(gs[0]),
                                               _ptr(gs[1]), _ptr(gs[2]), _ptr(grad_x)),
                   self.h)
        return grad_x

    def plv_group_create(self, problems, plv=True, iplv=True, ciplv=True,
                         C=False, diag=False):
        """Plan a grouped run.  `problems`: list of dicts with keys P,
        batch, N, T, optionally the input x (batch, N, T) for
        plv_analytic_grouped, and output tensors (plv, iplv, ciplv, C, diag);
        missing outputs are allocated here.  Returns a Group (keeps the
        tensors)."""
        mask = ((PLV_OUT_PLV if plv else 0) | (PLV_OUT_IPLV if iplv else 0) |
                (PLV_OUT_CIPLV if ciplv else 0) | (PLV_OUT_C if C else 0))
        arr = (_lib.PlvProblem * len(problems))()
        keep = []
        for k, q in enumerate(problems):
            B, N = q["batch"], q["N"]
            for key, want, shape, dt in (("plv", plv, (B, N, N), torch.float32),
                                         ("iplv", iplv, (B, N, N), torch.float32),
                                         ("ciplv", ciplv, (B, N, N), torch.float32),
                                         ("C", C, (B, N, N), torch.complex64),
                                         ("diag", diag, (B,), torch.float64)):
                if want and key not in q:
                    q[key] = torch.empty(shape, dtype=dt, device=self.device)
            x = q.get("x")
            xptr, ldx, xdt = None, 0, 0
            if x is not None:
                assert x.is_cuda and x.dim() == 3 and x.shape == (B, N, q["T"])
                if not (x.stride(-1) == 1 and
                        (N == 1 or x.stride(0) == N * x.stride(1))):
                    x = q["x"] = x.contiguous()
                xptr = x.data_ptr()
                ldx = x.stride(1) if N > 1 else max(x.stride(0), q["T"])
                xdt = _dtype_code(x)
            arr[k] = _lib.PlvProblem(
                q["P"].data_ptr(), B, N, q["T"],
                q["plv"].data_ptr() if plv else None,
                q["iplv"].data_ptr() if iplv else None,
                q["ciplv"].data_ptr() if ciplv else None,
                q["C"].data_ptr() if C else None,
                q["diag"].data_ptr() if diag else None,
                xptr, ldx, xdt)
            keep.append(q)
        g = ctypes.c_void_p()
        _lib.check(self.lib.plv_group_create(self.h, arr, len(problems), mask,
                                             ctypes.byref(g)), self.h)
        return Group(self, g, keep)

    def plv_analytic_grouped(self, group):
        """Eq. 3 + 4 for every problem of the plan that has an input x."""
        _lib.check(self.lib.plv_analytic_grouped(self.h, _stream(self.device),
                                                 group.g), self.h)
        return group.problems

    def plv_gram_grouped(self, group):
        _lib.check(self.lib.plv_gram_grouped(self.h, _stream(self.device),
                                             group.g), self.h)
        return group.problems

    def plv_group_tune(self, group, reps=3):
        """Autotune the plan's launch shapes (thread class per transform
        length, CTAs per SM, Gram tile schedule and split K) by timing
        candidates on its own buffers; returns what was chosen and measured
        as a dict."""
        r = _lib.PlvTuneResult()
        _lib.check(self.lib.plv_group_tune(self.h, _stream(self.device),
                                           group.g, int(reps),
                                           ctypes.byref(r)), self.h)
        out = {name: getattr(r, name) for name, _ in r._fields_}
        out["k1_per_sm"] = list(r.k1_per_sm)
        out["gram_schedule"] = ("longest_first", "balanced_rounds")[
            r.gram_schedule]
        return out

    def plv_group_configure(self, group, k1_widen=False, k1_per_sm=None,
                            gram_schedule="longest_first", gram_tile_cost=0,
                            gram_split=0):
        """Pin one of the tuner's candidate launch shapes without timing."""
        ps = (ctypes.c_int * 4)(*(k1_per_sm or (0, 0, 0, 0)))
        sched = {"longest_first": 0, "balanced_rounds": 1}[gram_schedule]
        _lib.check(self.lib.plv_group_configure(
            self.h, _stream(self.device), group.g, int(bool(k1_widen)), ps,
            sched, int(gram_tile_cost), int(gram_split)), self.h)

    def plv_trial_operands(self, V, E, N, ldv, l0, L, mode="asis", P=None):
        """Operands of the Gram over trials (Eq. 1 / 8 with mode "asis",
        Eq. 12 with mode "rms") from FP32 planar rows V [E][N][2][ldv]:
        columns l0 .. l0+L-1 become L problems of N rows and E samples."""
        assert V.is_cuda and V.dtype == torch.float32 and V.is_contiguous()
        assert V.numel() >= E * N * 2 * ldv
        if P is None:
            P = self.empty_phasors(L, N, E)
        m = {"asis": _lib.PLV_TRIAL_ASIS, "rms": _lib.PLV_TRIAL_RMS}[mode]
        _lib.check(self.lib.plv_trial_operands(self.h, _stream(self.device),
                                               _ptr(V), E, N, ldv, l0, L, m,
                                               _ptr(P)), self.h)
        return P

    def _fp32(self):
        """This handle if it is FP32, else an FP32 handle on the same device
        (for FP32 planar per-trial values)."""
        if self.precision == PLV_PREC_FP32:
            return self
        if getattr(self, "_h32", None) is None:
            self._h32 = Handle("fp32", device=self.device.index, checked=self.checked)
        return self._h32

    def time_resolved(self, x, l0=0, L=None, C=False, out=None):
        """Time-resolved PLV, iPLV, ciPLV over trials (Eq. 1 / 8, 13, 14) of
        x (E trials, N, T) at samples l0 .. l0+L-1: dict of (L, N, N)."""
        E, N, T = x.shape
        L = T - l0 if L is None else L
        if l0 < 0 or L < 0 or l0 + L > T:
            raise PlvError(_lib.PLV_ERR_INVALID, "samples out of range")
        V = self._fp32().plv_analytic(x)
        P = self.plv_trial_operands(V, E, N, phasor_ld(T), l0, L, "asis")
        return self.plv_gram(P, L, N, E, C=C, out=out)

    def plv_dft_bins(self, x, f0, F, X=None):
        """DFT of the real rows of x (..., T) at bins f0 .. f0+F-1, as FP32
        planar rows (..., 2, ld(F)) on the device."""
        assert x.is_cuda and x.dim() >= 1
        T = x.shape[-1]
        xs = x.reshape(-1, T)
        if xs.stride(-1) != 1:
            xs = xs.contiguous()
        rows = xs.shape[0]
        ldX = phasor_ld(F)
        if X is None:
            X = torch.empty(x.shape[:-1] + (2, ldX), dtype=torch.float32, device=x.device)
        _lib.check(self.lib.plv_dft_bins(self.h, _stream(self.device), _ptr(xs),
                                         _dtype_code(xs), rows, T, xs.stride(0),
                                         f0, F, _ptr(X), ldX), self.h)
        return X

    def coherency_bins(self, x, f0, F, C=False, out=None):
        """Coherency across trials (Eq. 12) of real x (E trials, N, T) at
        DFT bins f0 .. f0+F-1, entirely on the device: coherence, imaginary
        coherency and lagged coherence under the keys plv, iplv, ciplv,
        each (F, N, N)."""
        E, N, T = x.shape
        V = self.plv_dft_bins(x, f0, F)
        P = self.plv_trial_operands(V, E, N, phasor_ld(F), 0, F, "rms")
        return self.plv_gram(P, F, N, E, C=C, out=out)

    def coherency(self, X, C=False, out=None):
        """Coherency across trials (Eq. 12) of per-trial complex values X
        (E, N, L) on the device: coherence |coh|, imaginary coherency
        |Im coh| and lagged coherence Im coh / sqrt(1 - Re coh^2) under the
        keys plv, iplv, ciplv, each (L, N, N)."""
        assert X.is_cuda and X.is_complex() and X.dim() == 3
        E, N, L = X.shape
        ldv = phasor_ld(L)
        V = torch.zeros((E, N, 2, ldv), dtype=torch.float32, device=X.device)
        V[:, :, 0, :L] = X.real
        V[:, :, 1, :L] = X.imag
        P = self.plv_trial_operands(V, E, N, ldv, 0, L, "rms")
        return self.plv_gram(P, L, N, E, C=C, out=out)

    def set_gram_raster(self, width: int = 0):
        """Tile order of the tensor-core Gram (plv_set_gram_raster): super-
        columns of ``width`` 128-row blocks; 0 restores the default."""
        _lib.check(self.lib.plv_set_gram_raster(self.h, int(width)), self.h)

    def check_status(self) -> int:
        """Checked builds: the source line of the first out-of-range access
        the kernels caught (and skipped) on this handle's device since the
        last call, 0 for none; always 0 on the unchecked build
        (plv_check_status)."""
        v = ctypes.c_int(0)
        _lib.check(self.lib.plv_check_status(self.h, _stream(self.device), ctypes.byref(v)),
                   self.h)
        return int(v.value)

    def memory_usage(self):
        """(current, peak) device bytes held by the handle itself
        (plv_memory_usage)."""
        cur, peak = ctypes.c_size_t(0), ctypes.c_size_t(0)
        _lib.check(self.lib.plv_memory_usage(self.h, ctypes.byref(cur), ctypes.byref(peak)),
                   self.h)
        return int(cur.value), int(peak.value)

    def set_wait_limit(self, ns: int = 0):
        """Bound of the tensor-core Gram's pipeline waits in nanoseconds
        (plv_set_wait_limit); 0 restores the default of 4 s."""
        _lib.check(self.lib.plv_set_wait_limit(self.h, int(ns)), self.h)

    def plv_sync_status(self) -> int:
        v = ctypes.c_int(0)
        _lib.check(self.lib.plv_sync_status(self.h, _stream(self.device),
                                            ctypes.byref(v)), self.h)
        return int(v.value)

    # ---- convenience ------------------------------------------------------
    def connectivity(self, x, C=False, diag=False, out=None, P=None):
        """Whole forward path on real x (E, N, T): analytic signal, phasors,
        Gram and read-outs.  Returns a dict of (E, N, N) tensors."""
        E, N, T = x.shape
        P = self.plv_analytic(x, P)
        res = self.plv_gram(P, E, N, T, C=C, diag=diag, out=out)
        return res


class Group:
    """A grouped-Gram plan (plv_group) and the tensors it runs on."""

    def __init__(self, handle, g, problems):
        self.handle = handle
        self.g = g
        self.problems = problems

    def close(self):
        if getattr(self, "g", None):
            self.handle.lib.plv_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Connectivity(torch.autograd.Function):
    """PLV, iPLV, ciPLV of x (batch, N, T) with a hand-written backward.
    recompute=True: forward saves x and C (not the analytic signal); backward
    recomputes the analytic signal from x inside plv_backward.
    recompute=False: forward keeps the phasors and 1/|z| of
    plv_analytic_save (20 bytes per sample on a BF16X3 handle, 12 on FP32)
    and backward skips the recompute (plv_backward_saved)."""

    @staticmethod
    def forward(ctx, x, handle, recompute):
        E, N, T = x.shape
        ctx.handle = handle
        ctx.x_dtype = x.dtype
        ctx.recompute = recompute
        if recompute:
            P = handle.plv_analytic(x.detach())
            res = handle.plv_gram(P, E, N, T, C=True)
            ctx.save_for_backward(x.detach(), res["C"])
        else:
            saved = handle.plv_analytic_save(x.detach())
            res = handle.plv_gram(saved["P"], E, N, T, C=True)
            ctx.saved = saved
            ctx.save_for_backward(res["C"])
        return res["plv"], res["iplv"], res["ciplv"]

    @staticmethod
    def backward(ctx, g_plv, g_iplv, g_ciplv):
        if ctx.recompute:
            x, C = ctx.saved_tensors
            g = ctx.handle.plv_backward(x, C, g_plv, g_iplv, g_ciplv)
        else:
            (C,) = ctx.saved_tensors
            g = ctx.handle.plv_backward_saved(ctx.saved, C, g_plv, g_iplv, g_ciplv)
            ctx.saved = None
        return g.to(ctx.x_dtype), None, None


def connectivity(x, handle=None, recompute=True):
    """Differentiable (PLV, iPLV, ciPLV) of real x (batch, N, T) on the GPU;
    gradients flow to x through the library's backward kernels.  With
    recompute=False the forward pass keeps the analytic signal's phasors for
    the backward pass instead of recomputing them (more memory, less time;
    FP32 and BF16X3 handles)."""
    if handle is None:
        handle = _default_handle(x.device)
    return _Connectivity.apply(x, handle, recompute)


def gram_split_plan(nkb, chunk, grid, split):
    """The split-K plan of grouped Grams (host only, no device): for tiles
    of nkb[i] 32-sample K blocks, `chunk` K blocks per summation chunk, a
    grid of `grid` CTAs and factor `split`, the number of parts each tile
    runs as (plv_gram_split_plan)."""
    lib = _lib.load()
    n = len(nkb)
    a = (ctypes.c_int * max(n, 1))(*[int(v) for v in nkb])
    out = (ctypes.c_int * max(n, 1))()
    _lib.check(lib.plv_gram_split_plan(a, n, int(chunk), int(grid), int(split), out),
               None, lib)
    return list(out[:n])


_handles = {}


def _default_handle(device):
    key = (device.index if device.index is not None
           else torch.cuda.current_device())
    if key not in _handles:
        _handles[key] = Handle(precision="fp32", device=key)
    return _handles[key]
