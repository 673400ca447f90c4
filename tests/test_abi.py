"""The C ABI library builds, loads and exports every function gn.h declares (CPU only).

No compute call is made here; argument validation that happens before any
CUDA call (bad equation, bad widths) is exercised because it needs no GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gn.h")


@pytest.fixture(scope="module")
def libgn():
    from paper_2509_14185_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gn_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gn_init", "gn_residual", "gn_jacobian", "gn_gradient", "gn_step", "gn_gram",
                     "gn_damped_solve", "gn_destroy", "gn_error_string", "gn_param_count"]:
        assert required in names


def test_library_exports_every_declared_symbol(libgn):
    for name in declared_functions():
        assert hasattr(libgn, name), name


def test_binding_covers_every_export(libgn):
    from paper_2509_14185_gb300 import gn
    for name in declared_functions():
        assert name in gn.EXPORTS, name


def test_error_strings(libgn):
    f = libgn.gn_error_string
    f.restype = ctypes.c_char_p
    f.argtypes = [ctypes.c_int]
    assert f(0) == b"ok"
    assert b"positive definite" in f(-5)
    assert f(12345) == b"unknown status"


def test_invalid_problem_rejected_before_any_cuda_call(libgn):
    from paper_2509_14185_gb300 import gn
    L = gn.lib()
    p = gn.gn_problem()
    p.equation = 7
    h = ctypes.c_void_p()
    assert L.gn_init(ctypes.byref(p), None, ctypes.byref(h)) == gn.GN_ERR_INVALID
    p.equation = gn._inputs.CCF
    p.n_layers = 2
    p.widths[0], p.widths[1], p.widths[2] = 2, 8, 1      # CCF is 1D: input width must be 1
    assert L.gn_init(ctypes.byref(p), None, ctypes.byref(h)) == gn.GN_ERR_INVALID
    p.widths[0] = 1
    p.hilbert_m = 7                                       # odd node count
    assert L.gn_init(ctypes.byref(p), None, ctypes.byref(h)) == gn.GN_ERR_INVALID
    assert L.gn_init(None, None, ctypes.byref(h)) == gn.GN_ERR_INVALID
    assert L.gn_destroy(None) == 0
