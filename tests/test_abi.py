"""The C-ABI library builds, loads and exports every symbol include/plv.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1710_08037_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "plv.h")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(plv_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = header_functions()
    for n in ("plv_create", "plv_destroy", "plv_analytic", "plv_gram",
              "plv_metrics", "plv_normalize", "plv_sync_status"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert sorted(_lib.SIGNATURES) == header_functions()


def test_phasor_layout_helpers(lib):
    """Pure host helpers: padded row length and operand bytes."""
    lib.plv_phasor_ld.restype = ctypes.c_int64
    lib.plv_phasor_ld.argtypes = [ctypes.c_int]
    assert lib.plv_phasor_ld(1) == 32
    assert lib.plv_phasor_ld(32) == 32
    assert lib.plv_phasor_ld(500) == 512
    assert lib.plv_phasor_ld(4096) == 4096
    lib.plv_phasor_bytes.restype = ctypes.c_size_t
    lib.plv_phasor_bytes.argtypes = [ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int]
    assert lib.plv_phasor_bytes(None, 30, 4096, 4096) == 30 * 4096 * 4096 * 8
    assert lib.plv_phasor_bytes(None, -1, 4, 4) == 0


def test_null_handle_is_rejected_without_a_device(lib):
    """Host-side validation runs before any CUDA call."""
    lib.plv_gram.restype = ctypes.c_int
    rc = lib.plv_gram(None, None, None, 1, 4, 4, 1, None, None, None, None,
                      None)
    assert rc == _lib.PLV_ERR_INVALID
    lib.plv_last_error.restype = ctypes.c_char_p
    assert b"NULL" in lib.plv_last_error(None)
    rc = lib.plv_create(None, 0, 0, ctypes.c_size_t(0))
    assert rc == _lib.PLV_ERR_INVALID


def _c_layout(tmp_path, ctype_name, names):
    """sizeof and offsetof of a struct of include/plv.h, by the C compiler."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")
    src = tmp_path / f"layout_{ctype_name}.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "plv.h"\n'
        "int main(void) {\n"
        f'  printf("%zu\\n", sizeof({ctype_name}));\n' +
        "".join(f'  printf("%zu\\n", offsetof({ctype_name}, {n}));\n' for n in names) +
        "  return 0;\n}\n")
    exe = tmp_path / f"layout_{ctype_name}"
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    return [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                           text=True).stdout.split()]


@pytest.mark.parametrize("ctype_name, mirror", [("plv_problem", _lib.PlvProblem),
                                                ("plv_tune_result", _lib.PlvTuneResult)])
def test_struct_layout_matches_header(tmp_path, ctype_name, mirror):
    """The ctypes mirrors of the header's structs have the C compiler's size
    and field offsets."""
    names = [f[0] for f in mirror._fields_]
    got = _c_layout(tmp_path, ctype_name, names)
    want = [ctypes.sizeof(mirror)] + [getattr(mirror, n).offset for n in names]
    assert got == want


def test_tuner_validates_on_the_host(lib):
    """The autotuner and the configuration call reject NULL plans and
    out-of-range values before any CUDA call."""
    f = lib.plv_group_tune
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p]
    assert f(None, None, None, 3, None) == _lib.PLV_ERR_INVALID
    g = lib.plv_group_configure
    g.restype = ctypes.c_int
    g.argtypes = ([ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                           ctypes.c_int])
    assert g(None, None, None, 0, None, 0, 0) == _lib.PLV_ERR_INVALID


def test_every_entry_point_validates_before_touching_a_device(lib):
    """Every status-returning entry point, called with a NULL handle (or,
    without one, an invalid size) and zero arguments, fails with
    PLV_ERR_INVALID from its host-side checks; the destroy calls accept
    NULL.  No CUDA call is made, so this runs without a GPU."""
    # plv_debug_fault(PLV_FAULT_NONE, 0) disarms: valid with all zeros
    ok_on_null = {"plv_destroy", "plv_group_destroy", "plv_debug_fault"}
    not_status = {"plv_last_error", "plv_get_precision", "plv_phasor_ld",
                  "plv_phasor_bytes", "plv_debug_fault_armed", "plv_build_checked"}
    for name, (res, args) in _lib.SIGNATURES.items():
        if name in not_status:
            continue
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
        zeros = [None if a is ctypes.c_void_p or isinstance(a, type(ctypes.POINTER(ctypes.c_int)))
                 else 0 for a in args]
        rc = f(*zeros)
        want = _lib.PLV_OK if name in ok_on_null else _lib.PLV_ERR_INVALID
        assert rc == want, (name, rc)
    lib.plv_get_precision.restype = ctypes.c_int
    lib.plv_get_precision.argtypes = [ctypes.c_void_p]
    assert lib.plv_get_precision(None) == _lib.PLV_PREC_FP32


def test_noalloc_backward_rejects_on_the_host(lib):
    """The allocation-free backward checks sizes, the supported lengths and
    its fixed scratch limit before any CUDA call."""
    name = "plv_backward_noalloc"
    res, args = _lib.SIGNATURES[name]
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: rejected first
    common = (None, fake, _lib.PLV_F32)
    # a length that is not a power of two in range: unsupported
    rc = f(*common, 1, 4, 300, 300, fake, None, None, None, fake)
    assert rc == _lib.PLV_ERR_UNSUPPORTED
    # more scratch than the fixed array holds
    rc = f(*common, 64, 4096, 8192, 8192, fake, None, None, None, fake)
    assert rc == _lib.PLV_ERR_INVALID
    lib.plv_last_error.restype = ctypes.c_char_p
    assert b"scratch" in lib.plv_last_error(None)


def test_no_cpu_path_without_a_gpu():
    """Without a CUDA device the binding refuses to run instead of falling
    back to the CPU (the oracle is never on the product path)."""
    import torch
    import paper_1710_08037_gb300 as plv
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(plv.PlvError):
        plv.Handle(precision="bf16x3")
    import subprocess
    import sys
    out = subprocess.run([sys.executable, "-c",
                          "import sys, paper_1710_08037_gb300; print('oracle' in sys.modules)"],
                         cwd=ROOT, capture_output=True, text=True, check=True)
    assert out.stdout.strip() == "False"


def test_fault_injection_arms_and_validates_on_the_host(lib):
    """plv_debug_fault arms one host-side fault (allocation, launch, or the
    tensor-core Gram's withheld copy) with a countdown, rejects unknown kinds
    and countdowns below 1, and disarms with PLV_FAULT_NONE; no CUDA call."""
    f = lib.plv_debug_fault
    f.restype, f.argtypes = ctypes.c_int, [ctypes.c_int, ctypes.c_int]
    g = lib.plv_debug_fault_armed
    g.restype, g.argtypes = ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]
    n = ctypes.c_int(-1)
    assert f(_lib.PLV_FAULT_ALLOC, 3) == _lib.PLV_OK
    assert g(ctypes.byref(n)) == _lib.PLV_FAULT_ALLOC and n.value == 3
    assert f(_lib.PLV_FAULT_LAUNCH, 0) == _lib.PLV_ERR_INVALID
    assert f(99, 1) == _lib.PLV_ERR_INVALID
    assert g(None) == _lib.PLV_FAULT_ALLOC  # a rejected call leaves it armed
    assert f(_lib.PLV_FAULT_STALL, 1) == _lib.PLV_OK
    assert g(ctypes.byref(n)) == _lib.PLV_FAULT_STALL and n.value == 1
    assert f(_lib.PLV_FAULT_NONE, 0) == _lib.PLV_OK
    assert g(ctypes.byref(n)) == _lib.PLV_FAULT_NONE and n.value == 0


@pytest.mark.parametrize("env,kind,count", [("alloc", 1, 1), ("alloc:4", 1, 4),
                                            ("launch:2", 2, 2), ("timeout", 3, 1),
                                            ("launch:0", 0, 0), ("bogus", 0, 0),
                                            ("alloc:x", 0, 0)])
def test_fault_injection_from_the_environment(env, kind, count):
    """PLV_FAULT, read when the library loads, arms the same faults; a
    malformed value arms nothing (checked in a fresh process)."""
    import subprocess
    import sys
    code = ("import ctypes, sys; from paper_1710_08037_gb300 import build; "
            "lib = ctypes.CDLL(build.build()); n = ctypes.c_int(-1); "
            "lib.plv_debug_fault_armed.argtypes = [ctypes.POINTER(ctypes.c_int)]; "
            "k = lib.plv_debug_fault_armed(ctypes.byref(n)); print(k, n.value)")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                         env=dict(os.environ, PLV_FAULT=env), check=True)
    assert out.stdout.split() == [str(kind), str(count)]


def test_checked_build_flag(lib):
    """The regular library reports itself as unchecked; its check query
    rejects a NULL handle before touching a device."""
    lib.plv_build_checked.restype = ctypes.c_int
    assert lib.plv_build_checked() == 0
    f = lib.plv_check_status
    f.restype, f.argtypes = ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_int)]
    v = ctypes.c_int(-1)
    assert f(None, None, ctypes.byref(v)) == _lib.PLV_ERR_INVALID
