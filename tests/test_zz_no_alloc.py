"""octen_compress_noalloc: the compression entry point for callers that cannot
allocate device memory (fixed device-memory budgets handed out by a host
framework, plugin hosts that forbid the CUDA allocator).  Called through the C ABI and checked
against octen_compress, the allocating entry point, with the same summary
tolerances as the parity tests (fp32 1e-5, bf16 5e-3 relative Frobenius per
replica), on two calls in a row: the shared static scratch keeps the previous
call's contents, so the second call must not depend on them.

This file is collected last on purpose (see its name)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp32": 1e-5, "bf16": 5e-3}


@pytest.fixture(scope="module")
def pkg():
    import paper_1807_01350_gb300 as p

    assert torch.cuda.is_available()
    p.lib()
    return p


def _inputs(I, J, P, Q, S, t, prec, seed):
    from synth import factors, projections, round_to, slice_batch, time_projection

    A, B, C = factors(I, J, t, 4, seed)
    X = slice_batch(A, B, C, 0, t, 0.01, seed)
    U, V = projections(I, J, P, Q, S, seed, prec)
    W = time_projection(t, P, Q, S, seed, 0)
    xdt = torch.float32 if prec == "fp32" else torch.bfloat16
    dev = lambda a, dt=torch.float32: torch.as_tensor(np.asarray(a, np.float32),
                                                      device="cuda").to(dt)
    return dev(round_to(X, "fp32"), xdt), dev(U), dev(V), dev(W)


def _cfg(pkg, I, J, P, Q, S, prec):
    return pkg._Config(I, J, 4, P, Q, S, 1, pkg.PREC[prec])


def _call(pkg, fn, cfg, X, U, V, W, Z):
    L = pkg.lib()
    return getattr(L, fn)(ctypes.byref(cfg), None, X.data_ptr(), X.shape[0], U.data_ptr(),
                          V.data_ptr(), W.data_ptr(), Z.data_ptr())


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("shape,prec", [
    ((152, 144, 3, 24, 4, 7), "fp32"),
    ((152, 144, 3, 24, 4, 7), "bf16"),
    # 20 slices of 1000 x 1000 do not fit the scratch at once: several chunks
    ((1000, 1000, 8, 100, 10, 20), "fp32"),
])
def test_noalloc_matches_allocating_entry_point_twice(pkg, shape, prec):
    I, J, P, Q, S, t = shape
    X, U, V, W = _inputs(I, J, P, Q, S, t, prec, seed=31)
    cfg = _cfg(pkg, I, J, P, Q, S, prec)
    Z_ref = torch.empty((P, Q, Q, Q), device="cuda")
    assert _call(pkg, "octen_compress", cfg, X, U, V, W, Z_ref) == 0
    for call in range(2):
        Z = torch.full((P, Q, Q, Q), float("nan"), device="cuda")
        assert _call(pkg, "octen_compress_noalloc", cfg, X, U, V, W, Z) == 0
        torch.cuda.synchronize()
        for p in range(P):
            assert _rel(Z[p], Z_ref[p]) < TOL[prec], (call, p, _rel(Z[p], Z_ref[p]))


def test_noalloc_rejects_oversized_shapes_and_host_buffers(pkg):
    # the 4000 x 4000, P = 16, Q = 256 projections alone exceed the scratch
    cfg = _cfg(pkg, 4000, 4000, 16, 256, 32, "bf16")
    d = torch.zeros(8, device="cuda")
    L = pkg.lib()
    st = L.octen_compress_noalloc(ctypes.byref(cfg), None, d.data_ptr(), 1, d.data_ptr(),
                                  d.data_ptr(), d.data_ptr(), d.data_ptr())
    assert st == 1
    X, U, V, W = _inputs(40, 32, 2, 8, 2, 3, "fp32", seed=32)
    cfg = _cfg(pkg, 40, 32, 2, 8, 2, "fp32")
    Zh = np.empty((2, 8, 8, 8), np.float32)
    st = L.octen_compress_noalloc(ctypes.byref(cfg), None, X.data_ptr(), 3, U.data_ptr(),
                                  V.data_ptr(), W.data_ptr(), Zh.ctypes.data)
    assert st == 1
