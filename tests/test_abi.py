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
    assert (o.k, o.ell, o.reorth, o.precision, o.maxit) == (10, 30, gkl.REORTH_DGKS, 0, 1000)
    assert (o.out_host, o.reserved0, o.block) == (0, 0, 0)
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
    assert lib.gkl_scores(None, None, 0) == gkl.ERR_ARG
    assert lib.gkl_sync(None) == gkl.ERR_ARG
    assert lib.gkl_grad(None, None, None, None, None, 0.0) == gkl.ERR_ARG


def test_struct_layouts_match_header():
    """The ctypes mirrors of gkl_opts and gkl_info have the C layout: field
    offsets as a C compiler lays out include/gkl.h (checked with gcc)."""
    import shutil
    import subprocess
    import tempfile
    from paper_1808_03374_gb300 import gkl
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not found")
    fields = {"gkl_opts": gkl.Opts, "gkl_info": gkl.Info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gkl.h"', "int main(void) {"]
    for cname, cls in fields.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.c")
        open(src, "w").write("\n".join(lines))
        exe = os.path.join(d, "layout")
        subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for cname, cls in fields.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_binding_checks_buffer_sizes_before_the_call():
    """The library takes every length from the handle, so the binding refuses a
    caller tensor of the wrong shape, dtype or memory kind before passing its
    pointer (else the library would read or write past its end)."""
    import torch
    from paper_1808_03374_gb300.gkl import _need_buffer
    _need_buffer(torch.zeros(7), (7,), torch.float32, False, "v")        # accepted
    _need_buffer(torch.zeros(3, 5, dtype=torch.float64), (3, 5), torch.float64)
    for t, args in [(torch.zeros(6), ((7,),)),                           # too short
                    (torch.zeros(8), ((7,),)),                           # too long
                    (torch.zeros(5, 3), ((3, 5),)),                      # transposed
                    (torch.zeros(7), ((7,), torch.float64)),             # wrong dtype
                    (torch.zeros(7), ((7,), None, True)),                # host where device is needed
                    (torch.zeros(5, 3).t(), ((3, 5),))]:                 # not contiguous
        with pytest.raises(ValueError):
            _need_buffer(t, *args)
