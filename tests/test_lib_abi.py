"""The C-ABI library builds, loads and exports every symbol include/hssnd.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hssnd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", src))
    return sorted(n for n in names if n not in {"defined", "sizeof"})


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    from paper_1508_07798_gb300 import build as b
    b.build()
    return ctypes.CDLL(b.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "nd_order" in names and "hss_factor" in names and "hss_apply" in names and "fgmres_solve" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    from paper_1508_07798_gb300 import build as b
    b.build()
    from paper_1508_07798_gb300 import hssnd
    assert set(_declared()) == set(hssnd.EXPORTED)


def test_option_defaults_without_gpu(lib):
    from paper_1508_07798_gb300 import hssnd
    o = hssnd.factor_opts()
    assert o.tol == 1e-6 and o.r0 == 32 and o.oversample == 10 and o.compress == 1 and o.tensor_cores == 0
    f = hssnd.fgmres_opts()
    hssnd._lib.fgmres_opts_default(ctypes.byref(f))
    assert f.restart == 30 and f.rtol == 1e-8


def test_null_arguments_rejected_without_gpu(lib):
    from paper_1508_07798_gb300 import hssnd
    lib2 = hssnd._lib
    out = ctypes.c_void_p()
    assert lib2.nd_order(None, None, None, None, ctypes.byref(out)) == hssnd.HSS_EINVAL
    assert b"null" in lib2.hss_last_error()
    assert lib2.hss_apply(None, 1, None, 1, None, 1, None) == hssnd.HSS_EINVAL
