"""Host-side checks of the C ABI (no GPU): the library builds for sm_103a, loads, exports every entry
point that include/ibmles.h declares, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2002_06206_gb300 import build
    build.build()
    from paper_2002_06206_gb300 import ibmles
    return ibmles


def header_functions():
    src = open(os.path.join(ROOT, "include", "ibmles.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:[a-z_0-9]+\s*\**\s+)+\**\s*([a-z_][a-z_0-9]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "return")))


def test_header_declares_the_boundary():
    names = header_functions()
    for n in ("ibm_classify", "ibm_setup", "les_step", "poisson_solve", "forces", "les_create",
              "les_destroy", "ibm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    lib = C.CDLL(L.LIB_PATH)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing
    assert sorted(L.exported_symbols()) == header_functions()


def test_invalid_arguments_are_rejected_without_a_device(L):
    lib = L.lib()
    g = L.make_grid(0, 4, 4)
    out = C.c_void_p()
    prm = L.Params(0.1, 0.1, (C.c_double * 3)(1, 0, 0), (C.c_int32 * 6)(1, 2, 3, 3, 3, 3), 1, 1, 0, 0,
                   1e-6, 100, 16, 1e-4, 1.9, 0, 2, 1.6, 0.0)
    assert lib.les_create(C.byref(g), C.byref(prm), None, C.byref(out)) == L.E_INVALID
    assert b"extent" in lib.ibm_last_error()
    g = L.make_grid(8, 8, 8)
    bad = L.Params(0.1, 0.1, (C.c_double * 3)(1, 0, 0), (C.c_int32 * 6)(0, 2, 3, 3, 3, 3), 1, 1, 0, 0,
                   1e-6, 100, 16, 1e-4, 1.9, 0, 2, 1.6, 0.0)
    assert lib.les_create(C.byref(g), C.byref(bad), None, C.byref(out)) == L.E_INVALID
    assert b"periodic" in lib.ibm_last_error()
    bad.bc[0] = 1
    bad.precision = 7
    assert lib.les_create(C.byref(g), C.byref(bad), None, C.byref(out)) == L.E_INVALID
    bad.precision = 0
    bad.precond = 1
    bad.mg_omega = 2.5
    assert lib.les_create(C.byref(g), C.byref(bad), None, C.byref(out)) == L.E_INVALID
    assert b"omega" in lib.ibm_last_error()
    big = L.make_grid(2048, 2048, 2048)
    assert lib.les_create(C.byref(big), C.byref(prm), None, C.byref(out)) == L.E_INVALID
    gp = L.GeomParams(1e-9, 0.0, 0, 0)
    nc = C.c_int64()
    assert lib.ibm_classify(C.byref(g), None, 5, C.byref(gp), None, None, None, None, 0, C.byref(nc), None, None,
                            0, None) == L.E_INVALID
    assert lib.les_num_faces(C.byref(g)) == L.num_faces(8, 8, 8)
    assert lib.ibm_classify_workspace_bytes(C.byref(g), 10) > 3 * 512 * 16
