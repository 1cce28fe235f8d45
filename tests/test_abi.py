"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/pxa.h declares; argument validation answers without touching a device."""
import ctypes
import os
import re

import pytest

from paper_2004_00546_gb300 import pxa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|void|const char\*)\s+(pxa_\w+)\s*\(", text, flags=re.M))
    return names


def test_header_declares_the_binding_exports():
    decl = declared_functions()
    assert decl, "no declarations parsed"
    assert decl == set(pxa.EXPORTS)


def test_library_exports_every_declared_symbol(pxa_lib):
    for name in declared_functions():
        assert hasattr(pxa_lib, name), name


def test_invalid_arguments_are_rejected_without_a_device(pxa_lib):
    L = pxa_lib
    assert L.pxa_set_operator(None, None) == pxa.ERR_INVALID
    assert L.pxa_set_time(None, 1.0, 10, pxa.CN, 1) == pxa.ERR_INVALID
    assert L.pxa_gradient(None, 0, None, None) == pxa.ERR_INVALID
    L.pxa_destroy(None)  # must be a no-op
    assert L.pxa_last_error(None) == b"null context"
    h = ctypes.c_void_p()
    assert L.pxa_create(ctypes.byref(h), 4096, None) == pxa.ERR_CUDA
    assert L.pxa_create(None, 0, None) == pxa.ERR_INVALID
