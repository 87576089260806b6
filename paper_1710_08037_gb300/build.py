"""Build the CUDA library in-tree: csrc/*.cu -> _build/libplv.so (sm_103a).

Each translation unit (and each variant of a multiply-compiled one) is
compiled in parallel by nvcc, then linked into one
shared library exporting the C ABI of include/plv.h.  No cmake, no torch
extension machinery: the library has no torch types in it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libplv.so")
# the checked variant (-DPLV_CHECKED=1: bounds conditions of the kernels'
# index computations tested at run time, failures recorded, not trapped)
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libplv_checked.so")


def _paths(checked: bool):
    return (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                  "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc",
              shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


# Sources compiled more than once, with different -D flags (object suffix,
# flags): k_fwd.cu and k_bands.cu hold the launchers of one (input type, task
# kind).
VARIANTS = {
    "k_fwd.cu": [(f"_{t}_{k}", [f"-DPLV_K1_F64={f64}", f"-DPLV_K1_KIND={k}"])
                 for f64, t in ((0, "f32"), (1, "f64")) for k in range(4)],
    # the multi-band transform: forward task kinds only
    "k_bands.cu": [(f"_{t}_{k}", [f"-DPLV_K1_F64={f64}", f"-DPLV_K1_KIND={k}"])
                   for f64, t in ((0, "f32"), (1, "f64")) for k in range(3)],
}


def _units(checked: bool = False):
    """(source, object, extra flags) of every compiler run."""
    out = []
    bdir = _paths(checked)[0]
    extra = ["-DPLV_CHECKED=1"] if checked else []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        name = os.path.basename(src)[:-3]
        for suffix, flags in VARIANTS.get(os.path.basename(src), [("", [])]):
            out.append((src, os.path.join(bdir, name + suffix + ".o"), flags + extra))
    return out


def _deps():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu"))) + sorted(
        glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(ROOT, "include", "plv.h"), __file__]


def up_to_date(checked: bool = False) -> bool:
    lib = _paths(checked)[1]
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Compile every .cu for sm_103a and link libplv.so (libplv_checked.so
    with checked=True); returns its path."""
    bdir, lib = _paths(checked)
    if not force and up_to_date(checked):
        return lib
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    units = _units(checked)

    def compile_one(unit):
        src, obj, flags = unit
        cmd = [nvcc, *NVFLAGS, *flags, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    workers = max(1, min(len(units), os.cpu_count() or 8, 16))
    # longest first: the K1 variants, then the rest
    order = sorted(units, key=lambda u: 0 if u[2] else 1)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, order))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [],
                checked="--checked" in sys.argv))
