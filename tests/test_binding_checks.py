"""The Python binding refuses arrays whose sizes do not match the context's
shapes (EINVAL) before it hands a pointer to the library, whose kernels read
exactly the declared number of elements behind each one.  No GPU: the
contexts here are binding objects without a device context behind them, so
any call that passed the checks would stop at the library's NULL-context
check."""
import ctypes

import numpy as np
import pytest

import paper_1807_01350_gb300 as pkg


@pytest.fixture(scope="module")
def lib():
    from paper_1807_01350_gb300 import build as B

    B.build()
    return pkg.lib()


def _octen(lib, I=12, J=10, R=3, P=2, Q=6, S=2, prec="fp32"):
    g = pkg.Octen.__new__(pkg.Octen)
    g._lib, g._h, g.prec = lib, ctypes.c_void_p(), prec
    g.I, g.J, g.R, g.P, g.Q, g.S = I, J, R, P, Q, S
    g.Qd = S + P * (Q - S)
    return g


def _octen_n(lib, dims=(5, 4, 3), R=2, P=2, Q=4, S=1):
    g = pkg.OctenN.__new__(pkg.OctenN)
    g._lib, g._h = lib, ctypes.c_void_p()
    g.dims, g.N = list(dims), len(dims) + 1
    g.R, g.P, g.Q, g.S = R, P, Q, S
    g.Qd = S + P * (Q - S)
    return g


def _raises(fn, what):
    with pytest.raises(pkg.OctenError) as e:
        fn()
    assert e.value.status == 1
    assert what in str(e.value), str(e.value)


def test_three_mode_sizes(lib):
    g = _octen(lib)
    I, J, R, Qd, t = g.I, g.J, g.R, g.Qd, 4
    z = lambda *s: np.zeros(s, np.float32)
    good = dict(X_old=z(t, I, J), U_all=z(I, Qd), V_all=z(J, Qd), W_old=z(t, Qd), A0=z(I, R),
                B0=z(J, R), C0=z(t, R))
    for name, bad in (("X_old", z(t, I, J + 1)), ("U_all", z(I, Qd - 1)), ("V_all", z(I, Qd)),
                      ("W_old", z(t + 1, Qd)), ("A0", z(I, R + 1)), ("B0", z(J + 1, R)),
                      ("C0", z(t - 1, R))):
        args = dict(good, **{name: bad})
        _raises(lambda: g.init(**args), name)
    _raises(lambda: g.init(**dict(good, A0=None)), "A0")
    _raises(lambda: g.append(z(t, I, J - 1), z(t, Qd)), "X_new")
    _raises(lambda: g.append(z(t, I, J), z(t, Qd + 1)), "W_new")
    _raises(lambda: g.append(z(t, I, J), None), "W_new")
    _raises(lambda: g.fit(z(t, I + 1, J)), "X_all")
    # a batch given as (t * I) x J rows has t * I slices of the wrong size
    _raises(lambda: g.append(z(t * I, J), z(t, Qd)), "X_new")
    # sizes right: the call reaches the library, which has no context here
    with pytest.raises(pkg.OctenError) as e:
        g.append(z(t, I, J), z(t, Qd))
    assert e.value.status == 1 and "X_new" not in str(e.value)


def test_factor_destinations_must_be_the_callers_fp32_buffers(lib):
    g = _octen(lib)
    A = np.zeros((g.I, g.R), np.float32)
    B = np.zeros((g.J, g.R), np.float32)
    _raises(lambda: g.factors_into(np.zeros((g.I, g.R), np.float64), B, None), "A")
    _raises(lambda: g.factors_into(A, np.zeros((g.R, g.J), np.float32).T, None), "B")
    _raises(lambda: g.factors_into(A, np.zeros((g.J + 1, g.R), np.float32), None), "B")


def test_many_streams_sizes(lib):
    gs = [_octen(lib), _octen(lib, I=20)]
    xs = [np.zeros((2, 12, 10), np.float32), np.zeros((2, 12, 10), np.float32)]
    ws = [np.zeros((2, gs[0].Qd), np.float32)] * 2
    _raises(lambda: pkg.append_many(gs, xs, ws), "X_new[1]")
    _raises(lambda: pkg.append_many(gs, xs[:1], ws), "per stream")


def test_stateless_compression_sizes(lib):
    I, J, P, Q, S, t = 9, 8, 2, 5, 1, 3
    Qd = S + P * (Q - S)
    z = lambda *s: np.zeros(s, np.float32)
    _raises(lambda: pkg.compress(I, J, P, Q, S, z(t, I, J), z(I, Qd), z(J, Qd), z(t + 1, Qd)),
            "W_all")
    _raises(lambda: pkg.compress(I, J, P, Q, S, z(t, J, J), z(I, Qd), z(J, Qd), z(t, Qd)), "X")


def test_n_mode_sizes(lib):
    g = _octen_n(lib)
    d, R, Qd, t = g.dims, g.R, g.Qd, 3
    z = lambda *s: np.zeros(s, np.float32)
    Us = [z(n, Qd) for n in d]
    A0s = [z(n, R) for n in d]
    _raises(lambda: g.init(z(t, *d), Us[:2], z(t, Qd), A0s, z(t, R)), "projections")
    _raises(lambda: g.init(z(t, 5, 4, 4), Us, z(t, Qd), A0s, z(t, R)), "X_old")
    _raises(lambda: g.init(z(t, *d), [Us[0], z(3, Qd), Us[2]], z(t, Qd), A0s, z(t, R)),
            "U_all[1]")
    _raises(lambda: g.init(z(t, *d), Us, z(t, Qd), [A0s[0], A0s[1], z(3, R + 1)], z(t, R)),
            "A0[2]")
    _raises(lambda: g.append(z(t, 5, 4), z(t, Qd)), "X_new")
    _raises(lambda: g.append(z(t, *d), z(t, Qd - 1)), "W_new")
    _raises(lambda: g.fit(z(t, 5, 4, 2)), "X_all")


def test_async_append_takes_arrays_as_they_are(lib):
    """octen_append_async reads its inputs after the call returns, so the
    binding refuses arrays it would have to convert (a converted copy would be
    freed first): wrong element type or non-contiguous.  Refused before the
    library is called (EINVAL)."""
    g = _octen(lib, prec="fp32")
    I, J, Qd, t = g.I, g.J, g.Qd, 3
    x64 = np.zeros((t, I, J), np.float64)
    _raises(lambda: g.append_async(x64, np.zeros((t, Qd), np.float32)), "X_new")
    xT = np.zeros((t, J, I), np.float32).transpose(0, 2, 1)
    _raises(lambda: g.append_async(xT, np.zeros((t, Qd), np.float32)), "X_new")
    w64 = np.zeros((t, Qd), np.float64)
    _raises(lambda: g.append_async(np.zeros((t, I, J), np.float32), w64), "W_new")
    bf = _octen(lib, prec="bf16")
    # a bf16 context takes bf16 slices; numpy has no bf16, so numpy is refused
    _raises(lambda: bf.append_async(np.zeros((t, I, J), np.float32),
                                    np.zeros((t, bf.Qd), np.float32)), "X_new")
    # right types: the call reaches the library, which has no context here
    with pytest.raises(pkg.OctenError) as e:
        g.append_async(np.zeros((t, I, J), np.float32), np.zeros((t, Qd), np.float32))
    assert e.value.status == 1 and "X_new" not in str(e.value)
