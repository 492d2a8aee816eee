"""octen_compress_noalloc: the compression entry point for callers that cannot
allocate device memory (fixed device-memory budgets handed out by a host
framework, plugin hosts that forbid the CUDA allocator).  Called through the C
ABI and checked, on two calls in a row, against the FP64 oracle's compression
and against octen_compress, the allocating entry point, with the summary
tolerances of the parity tests (fp32 1e-5, bf16 5e-3, fp8 6e-2 relative
Frobenius per replica).  The shared static scratch keeps the previous call's
contents, so the second call must not depend on them.

This file is collected last on purpose (see its name)."""
import ctypes

import numpy as np
import pytest

import oracle
from tests._cases import Case, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp32": 1e-5, "bf16": 5e-3, "fp8": 6e-2}


@pytest.fixture(scope="module")
def pkg():
    import paper_1807_01350_gb300 as p

    assert torch.cuda.is_available()
    p.lib()
    return p


def _inputs(I, J, P, Q, S, t, prec, seed):
    """Device copies of a seeded case's slices (bf16 unless fp32) and rounded
    projections, and the same values as float64 for the oracle."""
    d = Case(I, J, 4, P, Q, S, t, (), 1, prec=prec, seed=seed).make()
    xdt = torch.float32 if prec == "fp32" else torch.bfloat16
    dev = lambda a, dt=torch.float32: torch.as_tensor(np.asarray(a, np.float32),
                                                      device="cuda").to(dt)
    return (dev(d["X"], xdt), dev(d["U"]), dev(d["V"]), dev(d["W"][0])), d


def _cfg(pkg, I, J, P, Q, S, prec):
    return pkg._Config(I, J, 4, P, Q, S, 1, pkg.PREC[prec])


def _call(pkg, fn, cfg, X, U, V, W, Z):
    L = pkg.lib()
    return getattr(L, fn)(ctypes.byref(cfg), None, X.data_ptr(), X.shape[0], U.data_ptr(),
                          V.data_ptr(), W.data_ptr(), Z.data_ptr())


@pytest.mark.parametrize("shape,prec", [
    ((152, 144, 3, 24, 4, 7), "fp32"),
    ((152, 144, 3, 24, 4, 7), "bf16"),
    ((152, 144, 3, 24, 4, 7), "fp8"),
    # 20 slices of 1000 x 1000 do not fit the scratch at once: several passes
    ((1000, 1000, 8, 100, 10, 20), "fp32"),
    # fp8: ~2.9 MB of scratch per slice, so 30 slices take two passes
    ((1024, 1024, 8, 100, 10, 30), "fp8"),
    # P = 2048 replicas of Q = 4: at most 65535 / P = 31 slices per pass (the
    # mode-1 grid limit), so 40 slices take two passes
    ((16, 16, 2048, 4, 1, 40), "fp32"),
])
def test_noalloc_matches_oracle_and_allocating_entry_point_twice(pkg, shape, prec):
    I, J, P, Q, S, t = shape
    (X, U, V, W), d = _inputs(I, J, P, Q, S, t, prec, seed=31)
    cfg = _cfg(pkg, I, J, P, Q, S, prec)
    Z_ref = torch.empty((P, Q, Q, Q), device="cuda")
    assert _call(pkg, "octen_compress", cfg, X, U, V, W, Z_ref) == 0
    Z_ref = Z_ref.cpu().numpy()
    Z_or = [oracle.compress(d["X"], oracle.replica_block(d["U"], p, Q, S),
                            oracle.replica_block(d["V"], p, Q, S),
                            oracle.replica_block(d["W"][0], p, Q, S)) for p in range(P)]
    for call in range(2):
        Z = torch.full((P, Q, Q, Q), float("nan"), device="cuda")
        assert _call(pkg, "octen_compress_noalloc", cfg, X, U, V, W, Z) == 0
        torch.cuda.synchronize()
        Z = Z.cpu().numpy()
        for p in range(P):
            assert rel(Z[p], Z_or[p]) < TOL[prec], (call, p, "oracle", rel(Z[p], Z_or[p]))
            assert rel(Z[p], Z_ref[p]) < TOL[prec], (call, p, "compress", rel(Z[p], Z_ref[p]))


def test_noalloc_rejects_oversized_shapes_bad_configs_and_host_buffers(pkg):
    L = pkg.lib()
    d = torch.zeros(8, device="cuda")
    # 4000 x 4000, P = 16, Q = 256, bf16: the transposed projections (62 MB)
    # plus one slice's mode-2 and mode-1 products (37 MB) exceed the 64 MiB
    cfg = _cfg(pkg, 4000, 4000, 16, 256, 32, "bf16")
    st = L.octen_compress_noalloc(ctypes.byref(cfg), None, d.data_ptr(), 1, d.data_ptr(),
                                  d.data_ptr(), d.data_ptr(), d.data_ptr())
    assert st == 1
    # outside octen_create's limits: P above the grid limit, R above 32
    for bad in (pkg._Config(16, 16, 4, 70000, 4, 1, 1, 0), pkg._Config(16, 16, 33, 2, 4, 1, 1, 0)):
        st = L.octen_compress_noalloc(ctypes.byref(bad), None, d.data_ptr(), 1, d.data_ptr(),
                                      d.data_ptr(), d.data_ptr(), d.data_ptr())
        assert st == 1
    (X, U, V, W), _ = _inputs(40, 32, 2, 8, 2, 3, "fp32", seed=32)
    cfg = _cfg(pkg, 40, 32, 2, 8, 2, "fp32")
    Zh = np.empty((2, 8, 8, 8), np.float32)
    st = L.octen_compress_noalloc(ctypes.byref(cfg), None, X.data_ptr(), 3, U.data_ptr(),
                                  V.data_ptr(), W.data_ptr(), Zh.ctypes.data)
    assert st == 1
