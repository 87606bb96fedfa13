"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h; argument checks that need no GPU return their status codes."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1201_6062_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(tdse_\w+)\s*\(", txt):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("tdse_create", "tdse_propagate", "tdse_norm", "tdse_populations", "tdse_adjoint",
                 "tdse_propagate_batch", "tdse_group_create", "tdse_group_propagate", "tdse_hmatvec"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_checks(lib):
    lib.tdse_create.restype = ctypes.c_int
    lib.tdse_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    E = (ctypes.c_double * 4)()
    # NULL out, bad sizes, missing dipoles: rejected before any CUDA call
    assert lib.tdse_create(E, None, 0, 4, 0, None) == 1
    assert lib.tdse_create(E, None, -1, 4, 0, ctypes.byref(out)) == 1
    assert b"lmax" in lib.tdse_last_error()
    assert lib.tdse_create(E, None, 0, 0, 0, ctypes.byref(out)) == 1
    assert lib.tdse_create(E, None, 0, 5000, 0, ctypes.byref(out)) == 1
    assert lib.tdse_create(E, None, 2, 4, 0, ctypes.byref(out)) == 1
    assert b"dipole" in lib.tdse_last_error()
    assert lib.tdse_create(E, None, 0, 4, 7, ctypes.byref(out)) == 1   # unknown precision
    assert lib.tdse_create(None, None, 0, 4, 0, ctypes.byref(out)) == 1
    assert out.value is None
    lib.tdse_propagate.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_double, ctypes.c_long] + \
        [ctypes.c_int] * 3 + [ctypes.c_void_p]
    assert lib.tdse_propagate(None, None, None, 1, 0.01, 1, 0, 4, 0, None) == 1
    assert lib.tdse_version() >= 10000


def test_gauge_argument_checks(lib):
    lib.tdse_set_gauge.restype = ctypes.c_int
    lib.tdse_set_gauge.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.tdse_set_gauge(None, 1) == 1
    f = lib.tdse_vector_potential_sin2
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_double] * 5 + [ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p]
    buf = (ctypes.c_double * 8)()
    assert f(0.1, 0.5, 10, 0.0, 0.01, 8, None, None) == 1                  # NULL output
    assert f(0.1, 0.0, 10, 0.0, 0.01, 8, buf, None) == 1                   # omega = 0
    assert f(0.1, 0.5, 10, 0.0, -0.01, 8, buf, None) == 1                  # h < 0
    assert f(0.1, 0.5, 10, -1.0, 0.01, 8, buf, None) == 1                  # t0 < 0
    assert f(0.1, 0.5, 10, 0.0, 0.01, 0, buf, None) == 1                   # no samples
    assert f(0.1, 0.5, 10, 1e9, 1e-3, 8, buf, None) == 1                   # t0/h too large
    assert f(float("nan"), 0.5, 10, 0.0, 0.01, 8, buf, None) == 1


def test_rkf45_argument_checks(lib):
    f = lib.tdse_propagate_rkf45
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_double] * 6 + [ctypes.c_long] + [ctypes.c_void_p] * 2
    assert f(None, None, None, 0.0, 1.0, 0.1, 1e-8, 0.0, 1.0, 10, None, None) == 1
