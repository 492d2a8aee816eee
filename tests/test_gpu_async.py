"""octen_append_async / octen_wait: appends enqueued without waiting, from
pinned host batches, each step's factors read back into pinned host buffers,
pipelined as a serving loop runs them (the next batch enqueued before the
previous one is waited for).  The results equal the same appends made with
octen_append, bit for bit, after every step."""
import numpy as np
import pytest

from tests._cases import Case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_1807_01350_gb300 as p

    assert torch.cuda.is_available()
    p.lib()
    return p


def _dev(a, dt=torch.float32):
    return torch.as_tensor(np.asarray(a, np.float32), device="cuda").to(dt)


def _pinned(a, dt=torch.float32):
    return torch.as_tensor(np.asarray(a, np.float32)).to(dt).pin_memory()


@pytest.mark.parametrize("prec,Q", [("bf16", 40), ("fp32", 12)])
def test_async_appends_equal_sync_appends(pkg, prec, Q):
    case = Case(160, 144, 5, 3, Q, 4, 8, (8, 6, 8, 8, 6), 6, prec=prec, seed=140)
    d = case.make()
    xdt = torch.float32 if prec == "fp32" else torch.bfloat16

    def start():
        g = pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters, prec,
                      stream=torch.cuda.current_stream())
        g.init(_dev(d["X"][:case.t_old], xdt), _dev(d["U"]), _dev(d["V"]), _dev(d["W"][0]),
               _dev(d["A0"]), _dev(d["B0"]), _dev(d["C0"]))
        return g

    bounds = np.cumsum((case.t_old,) + case.batches)
    # synchronous appends: the factors after every step
    ref = start()
    want = []
    for b, t in enumerate(case.batches):
        ref.append(_dev(d["X"][bounds[b]:bounds[b + 1]], xdt), _dev(d["W"][b + 1]))
        want.append(ref.factors())
    Y_ref = ref.replicas()
    ref.close()

    g = start()
    xs = [_pinned(d["X"][bounds[b]:bounds[b + 1]], xdt) for b in range(len(case.batches))]
    ws = [_pinned(d["W"][b + 1]) for b in range(len(case.batches))]
    outs = [(_pinned(np.zeros((case.I, case.R))), _pinned(np.zeros((case.J, case.R))),
             _pinned(np.zeros((t, case.R)))) for t in case.batches]
    tickets = []
    for b in range(len(case.batches)):
        tickets.append(g.append_async(xs[b], ws[b], *outs[b]))
        if b > 0:
            g.wait(tickets[b - 1])
    g.wait(tickets[-1])
    g.wait(tickets[0])                   # already waited for: fine
    with pytest.raises(pkg.OctenError) as e:
        g.wait(tickets[-1] + 1)          # never issued
    assert e.value.status == 1
    assert g.rows == bounds[-1]
    for b, (A, B, C) in enumerate(want):
        Ao, Bo, Co = (o.numpy() for o in outs[b])
        assert np.array_equal(Ao, A) and np.array_equal(Bo, B), b
        assert np.array_equal(Co, C[bounds[b]:bounds[b + 1]]), b
    A, B, C = g.factors()
    assert np.array_equal(C, want[-1][2])
    assert np.array_equal(g.replicas(), Y_ref)
    g.close()


def test_async_append_refuses_converted_inputs(pkg):
    case = Case(64, 48, 3, 2, 8, 2, 4, (4,), 3, prec="bf16", seed=141)
    d = case.make()
    g = pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters, "bf16")
    g.init(_dev(d["X"][:4], torch.bfloat16), _dev(d["U"]), _dev(d["V"]), _dev(d["W"][0]),
           _dev(d["A0"]), _dev(d["B0"]), _dev(d["C0"]))
    with pytest.raises(pkg.OctenError) as e:     # fp32 slices for a bf16 context
        g.append_async(_dev(d["X"][4:8]), _dev(d["W"][1]))
    assert e.value.status == 1 and "X_new" in str(e.value)
    assert g.rows == 4
    g.close()


def test_async_appends_grow_c_while_in_flight(pkg):
    """C outgrows its first 1024 rows while appends are in flight (two deep;
    32 slices per batch, fewer than the Qd = 60 distinct time-projection
    columns the new rows of C are solved from): the rows so far are copied on
    the stream and the old buffer is kept until nothing is in flight.  Every step's factors and new rows, and the final
    C, equal the synchronous appends' bit for bit, and once the last ticket
    has been waited for the context holds as much device memory as the
    synchronous one."""
    case = Case(64, 64, 3, 2, 32, 4, 8, (32,) * 32, 3, prec="bf16", seed=142)
    d = case.make()
    xdt = torch.bfloat16

    def start():
        g = pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters, "bf16",
                      stream=torch.cuda.current_stream())
        g.init(_dev(d["X"][:case.t_old], xdt), _dev(d["U"]), _dev(d["V"]), _dev(d["W"][0]),
               _dev(d["A0"]), _dev(d["B0"]), _dev(d["C0"]))
        return g

    bounds = np.cumsum((case.t_old,) + case.batches)
    n = len(case.batches)
    xs = [_pinned(d["X"][bounds[b]:bounds[b + 1]], xdt) for b in range(n)]
    ws = [_pinned(d["W"][b + 1]) for b in range(n)]
    ref = start()
    want = []
    for b in range(n):
        ref.append(xs[b], ws[b])   # the same host path (staging buffers) as below
        want.append(ref.factors())
    assert ref.rows > 1024
    ref_bytes = ref.device_bytes
    ref.close()

    g = start()
    outs = [(_pinned(np.zeros((case.I, case.R))), _pinned(np.zeros((case.J, case.R))),
             _pinned(np.zeros((32, case.R)))) for _ in range(n)]
    tickets = []
    for b in range(n):
        tickets.append(g.append_async(xs[b], ws[b], *outs[b]))
        if b >= 2:
            g.wait(tickets[b - 2])
    for tk in tickets[-2:]:
        g.wait(tk)
    assert g.rows == bounds[-1]
    for b, (A, B, C) in enumerate(want):
        Ao, Bo, Co = (o.numpy() for o in outs[b])
        assert np.array_equal(Ao, A) and np.array_equal(Bo, B), b
        assert np.array_equal(Co, C[bounds[b]:bounds[b + 1]]), b
    assert np.array_equal(g.factors()[2], want[-1][2])
    assert g.device_bytes == ref_bytes
    g.close()
