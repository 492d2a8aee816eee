"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/octen.h declares (no compute calls: they need a GPU)."""
import ctypes
import os
import re

import pytest

import paper_1807_01350_gb300 as pkg
from paper_1807_01350_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(octen_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    return B.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("octen_create", "octen_init", "octen_append", "octen_get_factors",
                     "octen_fit", "octen_destroy", "octen_compress"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_loads_library(built):
    L = pkg.lib()
    assert L.octen_status_name(1) == b"OCTEN_EINVAL"
    assert L.octen_last_error(None) == b"no context"


def test_create_rejects_bad_shapes_before_touching_the_device(built):
    # validation happens on the host: no GPU call is made for invalid configs
    cfg = pkg._Config(10, 10, 40, 2, 8, 2, 5, 0)      # R = 40 > 32
    h = ctypes.c_void_p()
    assert pkg.lib().octen_create(ctypes.byref(cfg), None, ctypes.byref(h)) == 1
    cfg = pkg._Config(10, 10, 4, 2, 8, 8, 5, 0)       # S = Q
    assert pkg.lib().octen_create(ctypes.byref(cfg), None, ctypes.byref(h)) == 1
