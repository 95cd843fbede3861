"""The C ABI library builds for sm_103a, loads without a GPU and exports every
function that include/aaomg.h and include/aaomg_stokes.h declare (no compute
call is made here)."""
import ctypes
import re

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1502_03917_gb300 import build

    build.build()
    import paper_1502_03917_gb300.aaomg as mg

    return mg


def test_exports_every_declared_function(lib):
    names = lib.header_functions()
    assert len(names) >= 14
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n


def test_binding_covers_header(lib):
    lib.load()
    for n in lib.header_functions():
        assert getattr(lib.load(), n).argtypes is not None, n


def test_options_layout_matches_header(lib):
    """The ctypes mirror of mg_options lists the header's fields in order with
    the same C types."""
    text = open(lib.HEADER).read()
    body = re.search(r"typedef struct mg_options \{(.*?)\} mg_options;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(int|double)\s+(\w+)\s*;", body)
    ctype = {"int": ctypes.c_int, "double": ctypes.c_double}
    assert [(n, ctype[t]) for t, n in fields] == [(n, t) for n, t in lib.Options._fields_]


def test_error_strings_without_device(lib):
    so = lib.load()
    assert so.mg_strerror(0) == b"ok"
    assert so.mg_strerror(-1) == b"bad argument"
    # argument validation happens before any device call
    opt = lib.Options()
    h = ctypes.c_void_p()
    assert so.mg_setup(0, 1.0, ctypes.byref(opt), ctypes.byref(h)) == lib.ERR_BAD_ARG
    assert so.mg_setup(5, -1.0, ctypes.byref(opt), ctypes.byref(h)) == lib.ERR_BAD_ARG
    assert b"alpha" in so.mg_last_error()


def test_no_oracle_on_product_path():
    """The product package never imports the oracle."""
    import os

    pkg = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1502_03917_gb300")
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(root, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, re.M), f
                assert "aaomg_oracle" not in text and "liboracle" not in text, f
                assert "stokes_oracle" not in text, f


def test_stokes_header_exported_and_bound(lib):
    from paper_1502_03917_gb300 import stokes

    names = stokes.header_functions()
    assert len(names) >= 11
    so = ctypes.CDLL(lib.LIB_PATH)
    stokes.load()
    for n in names:
        assert hasattr(so, n), n
        assert getattr(lib.load(), n).argtypes is not None, n


def test_stokes_options_layout_matches_header(lib):
    from paper_1502_03917_gb300 import stokes

    text = open(stokes.HEADER).read()
    body = re.search(r"typedef struct \{(.*?)\} ms_options;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(int|double)\s+(\w+)\s*;", body)
    ctype = {"int": ctypes.c_int, "double": ctypes.c_double}
    assert [(n, ctype[t]) for t, n in fields] == [(n, t) for n, t in stokes.Options._fields_]


def test_stokes_argument_errors_without_device(lib):
    from paper_1502_03917_gb300 import stokes

    so = stokes.load()
    h = ctypes.c_void_p()
    opt = stokes.Options()
    assert so.ms_setup(0, 1.0, ctypes.byref(opt), ctypes.byref(h)) == lib.ERR_BAD_ARG
    assert so.ms_setup(10, 1.0, ctypes.byref(opt), ctypes.byref(h)) == lib.ERR_BAD_ARG
    assert so.ms_setup(4, 0.0, None, ctypes.byref(h)) == lib.ERR_BAD_ARG
    assert b"alpha" in so.mg_last_error()
    opt.smoother = 7
    assert so.ms_setup(4, 1.0, ctypes.byref(opt), ctypes.byref(h)) == lib.ERR_BAD_ARG
    assert so.ms_sizes(None, 1, (ctypes.c_int * 4)()) == lib.ERR_BAD_ARG
