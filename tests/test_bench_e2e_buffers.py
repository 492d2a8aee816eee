"""The end-to-end leg of the benchmark reads the factors back into host
buffers sized once for the stream's final row count.  The binding accepts a C
of exactly the context's current rows, so the leg must hand it the leading
rows only.  No GPU: the binding object here sits on a stub library that
counts rows the way octen_rows does and answers octen_get_factors with OK;
the size checks run as they do on a real context."""
import numpy as np
import pytest

import bench
import paper_1807_01350_gb300 as pkg


class _StubLib:
    """octen_rows / octen_get_factors / octen_last_error of a context whose
    row count grows by a batch per append."""

    def __init__(self, rows):
        self.rows = rows
        self.calls = []

    def octen_rows(self, h):
        return self.rows

    def octen_get_factors(self, h, A, B, C, k_ref):
        self.calls.append(self.rows)
        k_ref._obj.value = self.rows
        return 0

    def octen_last_error(self, h):
        return b"stub"


def _octen(lib, I=40, J=36, R=5):
    g = pkg.Octen.__new__(pkg.Octen)
    g._lib, g._h, g.prec = lib, None, "bf16"
    g.I, g.J, g.R = I, J, R
    return g


def test_readback_buffers_sized_for_the_final_rows_pass_the_binding_checks():
    t_old, t, warmup, steps = 64, 16, 5, 20
    lib = _StubLib(t_old)
    g = _octen(lib)
    K_end = t_old + (warmup + steps) * t
    Ah = np.zeros((g.I, g.R), np.float32)
    Bh = np.zeros((g.J, g.R), np.float32)
    Ch = np.zeros((K_end, g.R), np.float32)
    # as bench.run_e2e: one read-back after every append, the rows growing
    for s in range(warmup + steps):
        lib.rows += t
        assert bench.read_factors(g, Ah, Bh, Ch) == lib.rows
    assert lib.calls == [t_old + (s + 1) * t for s in range(warmup + steps)]
    assert lib.calls[-1] == K_end


def test_the_whole_final_size_buffer_is_refused_before_the_last_append():
    lib = _StubLib(80)
    g = _octen(lib)
    Ch = np.zeros((96, g.R), np.float32)
    with pytest.raises(pkg.OctenError) as e:
        g.factors_into(np.zeros((g.I, g.R), np.float32), np.zeros((g.J, g.R), np.float32), Ch)
    assert e.value.status == 1 and "C" in str(e.value)
    assert not lib.calls
