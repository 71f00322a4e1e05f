"""CPU checks of the CUDA library: it builds for sm_103a, loads, and exports every entry point
that include/hodlr_qr.h declares; the binding covers them; the product package never reaches
the oracle.  No GPU calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hodlr_qr.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hodlr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1809_10585_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hodlr_build", "hodlr_qr", "hodlr_apply_q", "hodlr_apply_qt", "hodlr_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1809_10585_gb300 import binding
    assert set(declared_functions()) == set(binding.SYMBOLS)


def test_strerror_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.hodlr_strerror.restype = ctypes.c_char_p
    assert lib.hodlr_strerror(0) == b"ok"
    assert b"rank" in lib.hodlr_strerror(3)


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1809_10585_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, re.M), f
