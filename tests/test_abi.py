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


def test_nmode_create_rejects_bad_shapes_before_touching_the_device(built):
    L = pkg.lib()
    h = ctypes.c_void_p()

    def cfg(N, dims, R=2, P=2, Q=4, S=1, iters=5):
        d = (ctypes.c_int64 * (pkg.MAX_MODES - 1))(*(list(dims) + [0] * (pkg.MAX_MODES - 1 - len(dims))))
        return pkg._NConfig(N, R, P, Q, S, iters, d)

    for c in (cfg(2, (10,)),                      # fewer than three modes
              cfg(7, (4, 4, 4, 4, 4)),            # more than six
              cfg(4, (10, 10, 10), R=33),          # rank above 32
              cfg(4, (10, 10, 10), Q=4, S=4),      # S = Q
              cfg(4, (10, 0, 10)),                 # an empty mode
              cfg(6, (8, 8, 8, 8, 8), P=64, Q=32)):  # summaries too large
        assert L.octen_n_create(ctypes.byref(c), None, ctypes.byref(h)) == 1
    assert L.octen_n_last_error(None) == b"NULL context"


def _checkpoint(tmp_path, name, magic, cfg, hdr):
    path = tmp_path / name
    hdr_arr = (ctypes.c_int64 * len(hdr))(*hdr)
    path.write_bytes(magic + bytes(cfg) + bytes(hdr_arr))
    return str(path).encode()


def test_load_rejects_bad_checkpoint_headers_before_touching_the_device(built, tmp_path):
    # every rejection below happens while reading the header, before a
    # context (and any device memory) exists
    L = pkg.lib()
    h = ctypes.c_void_p()
    cfg = pkg._Config(100, 100, 5, 4, 20, 5, 50, 0)
    assert L.octen_load(str(tmp_path / "missing.bin").encode(), None, ctypes.byref(h)) == 1
    for name, magic, hdr in (
            ("magic.bin", b"OCTENXX1", [80, 0, 0, 0]),          # not a checkpoint
            ("rows0.bin", b"OCTENST1", [0, 0, 0, 0]),           # no rows of C
            ("rowsneg.bin", b"OCTENST1", [-5, 0, 0, 0]),
            ("rowsbig.bin", b"OCTENST1", [1 << 62, 0, 0, 0])):  # beyond any device
        assert L.octen_load(_checkpoint(tmp_path, name, magic, cfg, hdr), None,
                            ctypes.byref(h)) == 1, name
    trunc = tmp_path / "short.bin"
    trunc.write_bytes(b"OCTENST1" + bytes(cfg)[:12])
    assert L.octen_load(str(trunc).encode(), None, ctypes.byref(h)) == 1
    assert not h.value


def test_nmode_load_rejects_bad_checkpoint_headers_before_touching_the_device(built, tmp_path):
    L = pkg.lib()
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * (pkg.MAX_MODES - 1))(100, 100, 100, 0, 0)
    cfg = pkg._NConfig(4, 5, 8, 10, 3, 50, d)
    rest = [0] * pkg.MAX_MODES
    assert L.octen_n_load(str(tmp_path / "missing.bin").encode(), None, ctypes.byref(h)) == 1
    for name, magic, hdr in (
            ("magic.bin", b"OCTENST1", [30, 0] + rest),          # the 3-mode format
            ("rows0.bin", b"OCTENNM1", [0, 0] + rest),
            ("rowsbig.bin", b"OCTENNM1", [1 << 62, 0] + rest)):
        assert L.octen_n_load(_checkpoint(tmp_path, name, magic, cfg, hdr), None,
                              ctypes.byref(h)) == 1, name
    assert not h.value


def test_create_rejects_replica_counts_beyond_the_launch_grid(built):
    # P is a grid dimension of the replica kernels (at most 65535 blocks)
    L = pkg.lib()
    h = ctypes.c_void_p()
    cfg = pkg._Config(1000, 1000, 2, 65536, 3, 2, 5, 0)
    assert L.octen_create(ctypes.byref(cfg), None, ctypes.byref(h)) == 1
    assert not h.value
    d = (ctypes.c_int64 * (pkg.MAX_MODES - 1))(10, 10, 0, 0, 0)
    ncfg = pkg._NConfig(3, 2, 65536, 2, 1, 5, d)
    assert L.octen_n_create(ctypes.byref(ncfg), None, ctypes.byref(h)) == 1
    assert not h.value
