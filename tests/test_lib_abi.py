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


STRUCTS = ["hss_bsr", "hss_mesh", "hss_nd_opts", "hss_factor_opts", "fgmres_opts", "fgmres_stats",
           "hss_tree_desc", "hss_factor_info"]


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes mirror has the header struct's size and field offsets (a C
    program compiled against include/hssnd.h prints them)."""
    import shutil
    import subprocess
    from paper_1508_07798_gb300 import hssnd
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hssnd.h"', 'int main(void) {']
    for s in STRUCTS:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in getattr(hssnd, s)._fields_:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                         text=True).stdout.splitlines())
    for s in STRUCTS:
        cls = getattr(hssnd, s)
        assert int(got[f"{s} size"]) == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s} {f}"]) == getattr(cls, f).offset, (s, f)


def test_factor_defaults_overwrite_every_field(lib):
    """hss_factor_opts_default sets every field, so a C caller's uninitialised
    struct gets r_init = NULL and the default cap policy."""
    from paper_1508_07798_gb300 import hssnd
    o = hssnd.hss_factor_opts()
    ctypes.memset(ctypes.byref(o), 0xA5, ctypes.sizeof(o))
    hssnd._lib.hss_factor_opts_default(ctypes.byref(o))
    assert o.r_init is None and o.cap_policy == 0 and o.autotune == 0 and o.keep_schur == 0 and o.seed == 0
    assert o.rmax == 96 and o.probe == 0
    assert hssnd.factor_opts(cap_policy="accept").cap_policy == 1


def test_new_entry_points_reject_null_arguments_without_gpu(lib):
    from paper_1508_07798_gb300 import hssnd
    L = hssnd._lib
    out = ctypes.c_void_p()
    assert L.ilu0_factor(None, None, ctypes.byref(out)) == hssnd.HSS_EINVAL
    assert L.ilu0_factor(None, None, None) == hssnd.HSS_EINVAL
    assert L.ilu0_apply(None, 1, None, 1, None, 1, None) == hssnd.HSS_EINVAL
    assert L.fgmres_solve_ilu0(None, None, 1, None, 1, None, 1, None, None, None) == hssnd.HSS_EINVAL
    assert L.hss_factor_apply_plan(None, 0, None, None) == -hssnd.HSS_EINVAL
    # a block size outside [1, 64] is refused before any device access
    bad = hssnd.hss_bsr(4, 65, 1, 1, 1)
    assert L.ilu0_factor(ctypes.byref(bad), None, ctypes.byref(out)) == hssnd.HSS_EINVAL
    assert b"block size" in L.hss_last_error()
    L.ilu0_destroy(None)
