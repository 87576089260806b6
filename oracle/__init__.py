"""FP64 CPU oracle for the reformulated Phase Locking Value.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product library never
imports this package and shares no code with it.

The arithmetic lives in ``plv_oracle.c`` (plain C, FP64, OpenMP over rows):
direct-DFT analytic signal (Section II.A, Eq. 3), phase extraction, the
original pairwise mean of exp(i(phi_i - phi_j)) (Eq. 2) and the read-outs PLV
(Eq. 7), iPLV (Eq. 13) and ciPLV (Eq. 14).  ``backward.py`` holds the gradient
references (central finite differences of this oracle, and a plain-torch FP64
autograd graph).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "plv_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, -O2, no fast-math, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d = ctypes.POINTER(ctypes.c_double)
            L = ctypes.c_long
            lib.oracle_analytic.argtypes = [d, L, L, L, d, d]
            lib.oracle_plv_pairwise_rows.argtypes = [
                d, d, L, L, ctypes.POINTER(ctypes.c_long), L, d, d, d, d, d]
            lib.oracle_plv_pairwise.argtypes = [d, d, L, L, d, d, d, d, d]
            lib.oracle_gram_direct.argtypes = [d, d, L, L, d, d]
            lib.oracle_metrics.argtypes = [d, d, L, d, d, d]
            lib.oracle_analytic_band.argtypes = [d, L, L, L, d, d, d]
            lib.oracle_analytic_band.restype = ctypes.c_int
            lib.oracle_plv_time_resolved.argtypes = [d, d, L, L, L, L, L, d, d,
                                                     d, d, d]
            lib.oracle_dft_bins.argtypes = [d, L, L, L, L, L, d, d]
            lib.oracle_coherency_trials.argtypes = [d, d, L, L, L, d, d, d, d, d]
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_max_threads.restype = ctypes.c_int
            for f in ("oracle_analytic", "oracle_plv_pairwise_rows",
                      "oracle_plv_pairwise", "oracle_gram_direct",
                      "oracle_metrics", "oracle_plv_time_resolved",
                      "oracle_dft_bins", "oracle_coherency_trials"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def threads() -> int:
    return int(_load().oracle_max_threads())


def analytic(x: np.ndarray) -> np.ndarray:
    """Analytic signal z = x + i H{x} of each row of real ``x`` (..., T), by
    direct DFT in FP64 (Eq. 3).  Returns complex128 of the same shape."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    shape = x.shape
    T = shape[-1]
    rows = int(np.prod(shape[:-1])) if len(shape) > 1 else 1
    x2 = x.reshape(rows, T)
    zr = np.empty((rows, T))
    zi = np.empty((rows, T))
    rc = _load().oracle_analytic(_p(x2), rows, T, T, _p(zr), _p(zi))
    if rc != 0:
        raise RuntimeError("oracle_analytic failed")
    return (zr + 1j * zi).reshape(shape)


def pairwise(z: np.ndarray, rows=None) -> dict:
    """Original pairwise definition (Eq. 2) on one analytic signal ``z``
    (N, T) complex.  Returns dict with c (complex), plv, iplv, ciplv for pairs
    (rows[r], j); ``rows`` defaults to all rows."""
    z = np.asarray(z)
    N, T = z.shape
    zr = np.ascontiguousarray(z.real, dtype=np.float64)
    zi = np.ascontiguousarray(z.imag, dtype=np.float64)
    if rows is None:
        rows = np.arange(N)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    nr = rows.shape[0]
    cr = np.empty((nr, N))
    ci = np.empty((nr, N))
    plv = np.empty((nr, N))
    iplv = np.empty((nr, N))
    ciplv = np.empty((nr, N))
    rp = rows.ctypes.data_as(ctypes.POINTER(ctypes.c_long))
    rc = _load().oracle_plv_pairwise_rows(_p(zr), _p(zi), N, T, rp, nr,
                                          _p(cr), _p(ci), _p(plv), _p(iplv),
                                          _p(ciplv))
    if rc != 0:
        raise RuntimeError("oracle_plv_pairwise_rows failed")
    return {"c": cr + 1j * ci, "plv": plv, "iplv": iplv, "ciplv": ciplv}


def gram_direct(z: np.ndarray) -> np.ndarray:
    """Reformulated definition (Eq. 5-7) as a plain FP64 loop; (N, N)
    complex.  Used only to check the paper's equivalence claim."""
    z = np.asarray(z)
    N, T = z.shape
    zr = np.ascontiguousarray(z.real, dtype=np.float64)
    zi = np.ascontiguousarray(z.imag, dtype=np.float64)
    cr = np.empty((N, N))
    ci = np.empty((N, N))
    rc = _load().oracle_gram_direct(_p(zr), _p(zi), N, T, _p(cr), _p(ci))
    if rc != 0:
        raise RuntimeError("oracle_gram_direct failed")
    return cr + 1j * ci


def metrics(c: np.ndarray) -> dict:
    """Read-outs PLV (Eq. 7), iPLV (Eq. 13, absolute) and ciPLV (Eq. 14) of
    complex values ``c``; ciPLV = 0 where (1 - Re c)(1 + Re c) <= 0."""
    c = np.asarray(c, dtype=np.complex128)
    cr = np.ascontiguousarray(c.real).ravel()
    ci = np.ascontiguousarray(c.imag).ravel()
    n = cr.shape[0]
    plv = np.empty(n)
    iplv = np.empty(n)
    ciplv = np.empty(n)
    rc = _load().oracle_metrics(_p(cr), _p(ci), n, _p(plv), _p(iplv),
                                _p(ciplv))
    if rc != 0:
        raise RuntimeError("oracle_metrics failed")
    return {"plv": plv.reshape(c.shape), "iplv": iplv.reshape(c.shape),
            "ciplv": ciplv.reshape(c.shape)}


def connectivity(x: np.ndarray) -> dict:
    """Whole path for one epoch: real x (N, T) -> analytic signal (Eq. 3) ->
    pairwise PLV / iPLV / ciPLV (Eq. 2, 13, 14) for all ordered pairs."""
    z = analytic(x)
    out = pairwise(z)
    out["z"] = z
    return out


def connectivity_pairs(x: np.ndarray, pairs_i, pairs_j) -> dict:
    """Sampled outputs of the whole path for one epoch: only the rows named
    in ``pairs_i`` / ``pairs_j`` get their analytic signal, then the pairwise
    definition is evaluated for each (i, j).  Cost scales with the sample,
    not with N."""
    pairs_i = np.asarray(pairs_i, dtype=np.int64)
    pairs_j = np.asarray(pairs_j, dtype=np.int64)
    need = np.unique(np.concatenate([pairs_i, pairs_j]))
    pos = {int(r): k for k, r in enumerate(need)}
    z = analytic(np.asarray(x)[need])
    c = np.empty(pairs_i.shape[0], dtype=np.complex128)
    # one pairwise call per distinct row i over the needed columns
    for i in np.unique(pairs_i):
        sel = np.nonzero(pairs_i == i)[0]
        res = pairwise(z, rows=[pos[int(i)]])
        cols = np.array([pos[int(j)] for j in pairs_j[sel]])
        c[sel] = res["c"][0, cols]
    out = metrics(c)
    diag = pairs_i == pairs_j
    out["iplv"][diag] = 0.0
    out["ciplv"][diag] = 0.0
    out["c"] = c
    return out


def time_resolved(z: np.ndarray, t0: int = 0, L=None) -> dict:
    """Time-resolved PLV (Eq. 1 / Eq. 8) of trials ``z`` (E, N, T) complex:
    for samples t0 .. t0+L-1 the mean over trials of exp(i (phi_i - phi_j)),
    with the read-outs.  Returns dict of (L, N, N) arrays (c complex)."""
    z = np.asarray(z)
    E, N, T = z.shape
    L = T - t0 if L is None else L
    zr = np.ascontiguousarray(z.real, dtype=np.float64)
    zi = np.ascontiguousarray(z.imag, dtype=np.float64)
    out = {k: np.empty((L, N, N)) for k in ("cr", "ci", "plv", "iplv", "ciplv")}
    rc = _load().oracle_plv_time_resolved(
        _p(zr), _p(zi), E, N, T, t0, L, _p(out["cr"]), _p(out["ci"]),
        _p(out["plv"]), _p(out["iplv"]), _p(out["ciplv"]))
    if rc != 0:
        raise RuntimeError("oracle_plv_time_resolved failed")
    return {"c": out["cr"] + 1j * out["ci"], "plv": out["plv"],
            "iplv": out["iplv"], "ciplv": out["ciplv"]}


def dft_bins(x: np.ndarray, f0: int, F: int) -> np.ndarray:
    """DFT of the real rows of ``x`` (..., T) at bins f0 .. f0+F-1, by the
    direct sum in FP64.  Returns complex128 (..., F)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    shape = x.shape
    T = shape[-1]
    rows = int(np.prod(shape[:-1])) if len(shape) > 1 else 1
    Xr = np.empty((rows, F))
    Xi = np.empty((rows, F))
    rc = _load().oracle_dft_bins(_p(x.reshape(rows, T)), rows, T, T, f0, F,
                                 _p(Xr), _p(Xi))
    if rc != 0:
        raise RuntimeError("oracle_dft_bins failed")
    return (Xr + 1j * Xi).reshape(shape[:-1] + (F,))


def coherency_trials(X: np.ndarray) -> dict:
    """Coherency across trials (Eq. 12) of ``X`` (E, N, L) complex, per
    column l: coh (complex), coherence |coh|, imaginary coherency |Im coh|
    and lagged coherence Im coh / sqrt(1 - Re coh^2), each (L, N, N)."""
    X = np.asarray(X)
    E, N, L = X.shape
    xr = np.ascontiguousarray(X.real, dtype=np.float64)
    xi = np.ascontiguousarray(X.imag, dtype=np.float64)
    out = {k: np.empty((L, N, N)) for k in ("cr", "ci", "coh", "icoh", "lcoh")}
    rc = _load().oracle_coherency_trials(
        _p(xr), _p(xi), E, N, L, _p(out["cr"]), _p(out["ci"]), _p(out["coh"]),
        _p(out["icoh"]), _p(out["lcoh"]))
    if rc != 0:
        raise RuntimeError("oracle_coherency_trials failed")
    return {"c": out["cr"] + 1j * out["ci"], "coh": out["coh"],
            "icoh": out["icoh"], "lcoh": out["lcoh"]}


def windows(z: np.ndarray, t0: int, W: int, hop: int, nw: int) -> dict:
    """Sliding-window PLV (Eq. 2 over the W samples of each window w < nw,
    starting at t0 + w hop) of one analytic signal z (N, T), by the pairwise
    definition on each window's samples.  Returns dict of (nw, N, N) arrays
    (c complex, plv, iplv, ciplv)."""
    z = np.asarray(z)
    res = [pairwise(z[:, t0 + w * hop: t0 + w * hop + W]) for w in range(nw)]
    return {k: np.stack([r[k] for r in res]) for k in ("c", "plv", "iplv", "ciplv")}


def analytic_band(x: np.ndarray, band: np.ndarray) -> np.ndarray:
    """Analytic signal of the band-passed rows of real x (..., T): the band
    mask (floor(T/2) + 1 real values on the bins 0 .. T/2) and the analytic
    mask in one transform, by direct DFT in FP64.  Complex128, x's shape."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    shape = x.shape
    T = shape[-1]
    band = np.ascontiguousarray(np.asarray(band, dtype=np.float64))
    assert band.shape == (T // 2 + 1,)
    rows = int(np.prod(shape[:-1])) if len(shape) > 1 else 1
    zr = np.empty((rows, T))
    zi = np.empty((rows, T))
    rc = _load().oracle_analytic_band(_p(x.reshape(rows, T)), rows, T, T, _p(band),
                                      _p(zr), _p(zi))
    if rc != 0:
        raise RuntimeError("oracle_analytic_band failed")
    return (zr + 1j * zi).reshape(shape)
