"""The C-ABI library loads and exports every entry point include/fedvr_negf.h
declares (no compute: these run without a GPU)."""
import ctypes as C
import os
import re

import pytest

from paper_0911_4348_gb300 import _native
from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "fedvr_negf.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_native.LIB_PATH):
        from paper_0911_4348_gb300 import build
        build.build()
    return _native.lib()


def test_header_declares_expected_calls():
    names = _declared()
    for must in ("build_fedvr", "set_potential", "solve_hf", "solve_2b", "fedvr_sigma2",
                 "fedvr_conv_sigma_g", "fedvr_conv_g0", "fedvr_power_mesh"):
        assert must in names


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = _declared()
    assert set(names) == set(_native.SIGNATURES), (set(names) ^ set(_native.SIGNATURES))
    for n in names:
        assert hasattr(lib, n), n


def test_null_context_is_rejected_without_touching_the_gpu(lib):
    nb = C.c_int()
    assert lib.build_fedvr(None, 4, 5, -1.0, 1.0, 0, C.byref(nb)) == -1
    assert lib.solve_hf(None, 100.0, 1e-12, 10, None, None) == -1
    assert lib.fedvr_sigma2(None, 4, 3, 2.0, None, None, None, 0) == -1
    assert lib.fedvr_create(None, None) == -1
    assert lib.fedvr_last_error(None) == b"null context"
    lib.fedvr_destroy(None)
