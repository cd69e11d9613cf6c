"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/gkl.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gkl_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1808_03374_gb300 import build, gkl
    build()
    return gkl.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gkl_init", "gkl_matvec", "gkl_rmatvec", "gkl_svd", "gkl_destroy", "gkl_colstats"):
        assert required in names


def test_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_match_header():
    from paper_1808_03374_gb300 import gkl
    assert sorted(gkl.EXPORTS) == [n for n in declared_functions() if n in gkl.EXPORTS]
    assert set(declared_functions()) <= set(gkl.EXPORTS) | {"gkl_grad"}


def test_host_only_entry_points(lib):
    from paper_1808_03374_gb300 import gkl
    assert b"sm_103a" in lib.gkl_version()
    o = gkl.Opts()
    lib.gkl_opts_default(ctypes.byref(o))
    assert (o.k, o.ell, o.reorth, o.precision, o.maxit) == (10, 30, 0, 0, 1000)
    assert o.tol == 1e-10 and o.v0 is None
    assert lib.gkl_last_error(None)


def test_argument_errors_without_device(lib):
    from paper_1808_03374_gb300 import gkl
    h = ctypes.c_void_p()
    # NULL packed buffer and bad stride are rejected before any device work
    assert lib.gkl_init(ctypes.byref(h), None, 10, 10, 16, None, None, None) == gkl.ERR_ARG
    assert b"NULL" in lib.gkl_last_error(None)
    fake = ctypes.c_void_p(4096)
    assert lib.gkl_init(ctypes.byref(h), fake, 100, 10, 8, None, None, None) == gkl.ERR_ARG
    assert lib.gkl_init(ctypes.byref(h), fake, 100, 10, 16, None, None, None) == gkl.ERR_ARG  # 16*4 < 100
    assert lib.gkl_svd(None, None, None, None, None, None, None) == gkl.ERR_ARG
    assert lib.gkl_matvec(None, 0, None, None) == gkl.ERR_ARG
