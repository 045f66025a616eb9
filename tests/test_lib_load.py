"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/mx.h (no compute calls: no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mx_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1908_03634_gb300 import build as b
    b.build()
    import paper_1908_03634_gb300 as mx
    return mx.load()


def test_every_declared_symbol_is_exported(lib):
    import paper_1908_03634_gb300 as mx
    decl = declared_symbols()
    assert "mx_mac_project" in decl and "mx_residual" in decl
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(mx.exported_symbols()) == sorted(decl)


def test_library_is_sm103a_only():
    from paper_1908_03634_gb300 import build as b
    assert "arch=compute_103a,code=sm_103a" in b.ARCH


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1908_03634_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "oracle.h" not in txt, f


def test_null_context_rejected_without_gpu(lib):
    import ctypes as C
    import paper_1908_03634_gb300 as mx
    g = mx.mx_geom()
    # NULL context: argument error, no device work
    assert lib.mx_mac_project(None, C.byref(g), None, None, None, None, None, None, None, None, None) == mx.MX_ERR_ARG
    o = mx.mx_opts()
    lib.mx_default_opts(C.byref(o))
    assert o.rel_tol == 1e-10 and o.prec == mx.MX_PREC_MIXED and o.nu1 == 2
