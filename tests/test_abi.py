"""The C-ABI library loads and exports every entry point include/*.h declares (no GPU
needed), and argument errors come back as status codes."""
import ctypes as ct
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(fc2d_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2010_03901_gb300.build import build, LIB
    build()
    return ct.CDLL(LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "fc2d_plan" in names and "fc2d_extend_coeffs" in names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_argument_errors_are_status_codes(lib):
    lib.fc2d_plan.restype = ct.c_int
    lib.fc2d_last_error.restype = ct.c_char_p
    out = ct.c_void_p()
    assert lib.fc2d_plan(None, None, None, ct.byref(out)) == 1  # FC2D_ERR_ARG
    assert b"null" in lib.fc2d_last_error()
    lib.fc2d_extend.restype = ct.c_int
    assert lib.fc2d_extend(None, 1, None, None, None, None) == 1
    lib.fc2d_wait_selftest.restype = ct.c_int
    lib.fc2d_wait_selftest.argtypes = [ct.c_void_p, ct.c_uint32, ct.c_void_p]
    assert lib.fc2d_wait_selftest(None, 16, None) == 1
    assert b"null plan" in lib.fc2d_last_error()


def test_binding_names_match_the_abi():
    from paper_2010_03901_gb300 import fc2d
    names = declared_symbols()
    methods = ({m for m in dir(fc2d.Plan) if m.startswith("fc2d_")} |
               {m for m in dir(fc2d.Group) if m.startswith("fc2d_")} |
               {"fc2d_plan", "fc2d_group_create", "fc2d_probe_fp64"})
    skip = {"fc2d_plan_info", "fc2d_last_error", "fc2d_fc_matrices_compute"}
    assert (names - skip) <= methods | {"fc2d_destroy"}, names - methods
