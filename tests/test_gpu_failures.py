"""Failure paths of the library, exercised without faulting or hanging the GPU.

* Bounded waits: the pipeline waits of the tensor-core GEMMs are given a budget
  of one clock cycle (OCTEN_WAIT_BUDGET_CYCLES, a debug setting), so they run
  out before their first operands land.  The kernels then raise the timeout
  flag, drain what they issued and free their tensor memory; the call returns
  OCTEN_ETIMEOUT promptly and the device stays usable.
* Numerical failure: all-zero slices make the replica summaries zero, so the
  first C update is zero and the next update's normal-equation matrix (a
  Hadamard product of Grams) is zero even after diagonal loading:
  OCTEN_ENUMERIC.
* Allocation failure: a device-memory limit (OCTEN_DEVICE_MEMORY_LIMIT) makes
  octen_create, or the first append's scratch allocation, fail with
  OCTEN_ENOMEM; the append leaves the state exactly as it was.
"""
import time

import numpy as np
import pytest

import oracle
from tests._cases import Case, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_1807_01350_gb300 as p

    assert torch.cuda.is_available()
    p.lib()
    return p


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a, np.float32), device="cuda").to(dtype)


def _context(pkg, case, d, X=None):
    g = pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters, case.prec,
                  stream=torch.cuda.current_stream())
    xdt = torch.float32 if case.prec == "fp32" else torch.bfloat16
    X = d["X"] if X is None else X
    g.init(dev(X[:case.t_old], xdt), dev(d["U"]), dev(d["V"]), dev(d["W"][0]), dev(d["A0"]),
           dev(d["B0"]), dev(d["C0"]))
    return g


def test_compression_wait_budget_runs_out(pkg, monkeypatch):
    I, J, P, Q, S, t = 152, 144, 3, 24, 4, 7   # both contractions on tcgen05
    case = Case(I, J, 4, P, Q, S, t, (), 1, prec="bf16", seed=41)
    d = case.make()
    args = (I, J, P, Q, S, dev(d["X"], torch.bfloat16), dev(d["U"]), dev(d["V"]),
            dev(d["W"][0]))
    monkeypatch.setenv("OCTEN_AUTOTUNE", "0")
    monkeypatch.setenv("OCTEN_WAIT_BUDGET_CYCLES", "1")
    n0 = pkg.tc_launch_count()
    t0 = time.perf_counter()
    with pytest.raises(pkg.OctenError) as e:
        pkg.compress(*args, prec="bf16")
    assert e.value.status == 4, str(e.value)          # OCTEN_ETIMEOUT
    assert time.perf_counter() - t0 < 30
    assert pkg.tc_launch_count() - n0 == 2
    # the normal budget again: the same call succeeds and is right
    monkeypatch.delenv("OCTEN_WAIT_BUDGET_CYCLES")
    Z = pkg.compress(*args, prec="bf16")
    for p in range(P):
        ref = oracle.compress(d["X"], oracle.replica_block(d["U"], p, Q, S),
                              oracle.replica_block(d["V"], p, Q, S),
                              oracle.replica_block(d["W"][0], p, Q, S))
        assert rel(Z[p], ref) < 5e-3


def test_append_wait_budget_runs_out_and_the_context_is_destroyed_cleanly(pkg, monkeypatch):
    # Q = 64, bf16: the compression and the replica CP-ALS run on tcgen05
    case = Case(96, 80, 4, 2, 64, 8, 8, (8, 8), 5, prec="bf16", seed=42)
    d = case.make()
    monkeypatch.setenv("OCTEN_AUTOTUNE", "0")
    g = _context(pkg, case, d)
    monkeypatch.setenv("OCTEN_WAIT_BUDGET_CYCLES", "1")
    t0 = time.perf_counter()
    with pytest.raises(pkg.OctenError) as e:
        g.append(dev(d["X"][8:16], torch.bfloat16), dev(d["W"][1]))
    assert e.value.status == 4, str(e.value)
    assert time.perf_counter() - t0 < 60
    assert g.rows == 8          # K is not advanced after ETIMEOUT
    g.close()
    monkeypatch.delenv("OCTEN_WAIT_BUDGET_CYCLES")
    # a fresh context on the same device updates normally
    g = _context(pkg, case, d)
    g.append(dev(d["X"][8:16], torch.bfloat16), dev(d["W"][1]))
    assert g.rows == 16
    o, ref = case.oracle_run(d, upto=1)
    Y = g.replicas()
    for p in range(case.P):
        assert rel(Y[p], ref[0]["Y"][p]) < 5e-3
    g.close()


@pytest.mark.parametrize("prec,Q", [("fp32", 12), ("fp32", 40), ("bf16", 64)])
def test_zero_slices_report_numeric_failure(pkg, prec, Q):
    # fp32 Q = 12: the single-launch small-replica ALS; fp32 Q = 40: the SIMT
    # passes; bf16 Q = 64: the tensor-core passes
    case = Case(96, 80, 3, 2, Q, 4, 6, (6,), 4, prec=prec, seed=43)
    d = case.make()
    zeros = np.zeros_like(d["X"])
    g = _context(pkg, case, d, X=zeros)
    xdt = torch.float32 if prec == "fp32" else torch.bfloat16
    with pytest.raises(pkg.OctenError) as e:
        g.append(dev(zeros[6:12], xdt), dev(d["W"][1]))
    assert e.value.status == 5, str(e.value)          # OCTEN_ENUMERIC
    assert "pivot" in str(e.value)
    assert g.rows == 6
    g.close()


def test_device_memory_limit_gives_enomem_and_leaves_the_state_unchanged(pkg, monkeypatch):
    case = Case(64, 56, 3, 2, 16, 4, 8, (8,), 4, prec="fp32", seed=44)
    d = case.make()
    X = dev(d["X"])
    # the memory a context holds after init, and after its first append
    g = _context(pkg, case, d)
    held_init = g.device_bytes
    g.append(X[8:16], dev(d["W"][1]))
    held_append = g.device_bytes
    g.close()
    assert 0 < held_init < held_append
    # below the state itself: create fails
    monkeypatch.setenv("OCTEN_DEVICE_MEMORY_LIMIT", str(held_init // 4))
    with pytest.raises(pkg.OctenError) as e:
        pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters, case.prec)
    assert e.value.status == 2                        # OCTEN_ENOMEM
    # room for the state, not for the append's scratch
    monkeypatch.setenv("OCTEN_DEVICE_MEMORY_LIMIT", str(held_init))
    g = _context(pkg, case, d)
    assert g.device_bytes == held_init
    A0, B0, C0 = g.factors()
    Y0 = g.replicas()
    with pytest.raises(pkg.OctenError) as e:
        g.append(X[8:16], dev(d["W"][1]))
    assert e.value.status == 2, str(e.value)
    assert g.rows == 8 and g.device_bytes <= held_init
    A1, B1, C1 = g.factors()
    assert np.array_equal(A0, A1) and np.array_equal(B0, B1) and np.array_equal(C0, C1)
    assert np.array_equal(Y0, g.replicas())
    g.close()
    # with room for it the same append goes through
    monkeypatch.setenv("OCTEN_DEVICE_MEMORY_LIMIT", str(held_append))
    g = _context(pkg, case, d)
    g.append(X[8:16], dev(d["W"][1]))
    assert g.rows == 16
    g.close()
