"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs, stage by stage (summaries, raw replica CP, anchor match,
lifted factors, fit).

Tolerances.  FP32: summaries within 1e-5 relative Frobenius error per
replica (fp32 FFMA accumulation over J and I terms); replica factors and the
lifted factors within 1e-3 (the lift operators are fp32 Cholesky solves whose
error grows with cond(U^T U)); fit within 1e-4; factor-match
score against the oracle's factors >= 0.999.  BF16: the mode-2 product is
rounded to bf16 before the mode-1 contraction, a relative error of about
2^-9 / sqrt(3) ~ 1.1e-3 per element that the two later contractions average but
do not remove: summaries within 5e-3, fit within 1e-3.  FP8: per-slice e4m3
quantisation of the slices has unit roundoff 2^-4, an RMS relative error of
about 3 % per element that random projections preserve (they keep norms, so
they do not average independent errors away): summaries within 6e-2.  That
error acts like three times the 1 % data noise, and an FP64 run of the
oracle on e4m3-quantised slices loses 1.7e-3 to 2.0e-3 of fit against the
unquantised oracle at every size tried (I = 100 .. 400): fit within 3e-3.
Factor-match score against the oracle >= 0.99 for both reduced paths.
"""
import numpy as np
import pytest

import oracle
from tests._cases import Case, rel
from tests._metrics import fms

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_1807_01350_gb300 as p

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    p.lib()
    return p


def dev(a, dtype=None):
    t = torch.as_tensor(np.asarray(a, np.float32), device="cuda")
    return t if dtype is None else t.to(dtype)


def slices(a, prec):
    return dev(a, torch.float32 if prec == "fp32" else torch.bfloat16)


def run_gpu(pkg, case, d, upto=None):
    g = pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters, case.prec)
    g.init(slices(d["X"][:case.t_old], case.prec), dev(d["U"]), dev(d["V"]), dev(d["W"][0]),
           dev(d["A0"]), dev(d["B0"]), dev(d["C0"]))
    k = case.t_old
    out = []
    for b, t in enumerate(case.batches[:upto]):
        g.append(slices(d["X"][k:k + t], case.prec), dev(d["W"][b + 1]))
        k += t
        A, B, C = g.factors()
        out.append(dict(Y=g.replicas(), A=A, B=B, C=C, raw=g.replica_factors(0),
                        hat=g.replica_factors(1),
                        fit=g.fit(slices(d["X"][:k], case.prec))))
    return g, out


TOL = {"fp32": dict(Y=1e-5, F=1e-3, fit=1e-4, fms=0.999),
       "bf16": dict(Y=5e-3, F=5e-2, fit=1e-3, fms=0.99),
       "fp8": dict(Y=6e-2, F=2e-1, fit=3e-3, fms=0.99)}


def check_update(case, d, gpu_states, ref_states, tol=None, X_fit=None):
    """GPU states against oracle states; the oracle's fit is taken on X_fit
    (default: the case's slices, the ones the GPU's fit is taken on)."""
    tol = tol or TOL[case.prec]
    X_fit = d["X"] if X_fit is None else X_fit
    k = case.t_old
    for b, (gs, rs) in enumerate(zip(gpu_states, ref_states)):
        k += case.batches[b]
        for p in range(case.P):
            assert rel(gs["Y"][p], rs["Y"][p]) < tol["Y"], ("Y", b, p, rel(gs["Y"][p], rs["Y"][p]))
        At, Bt, Ct, perm, scales = gs["raw"]
        for p in range(case.P):
            ra, rb, rc = rs["raw"][p]
            for name, x, y in (("At", At[p], ra), ("Bt", Bt[p], rb), ("Ct", Ct[p], rc)):
                assert rel(x, y) < tol["F"], (name, b, p, rel(x, y))
        Ah, Bh, Ch, perm, scales = gs["hat"]
        for p in range(case.P):
            assert np.array_equal(perm[p], rs["hat"][p][3]), ("perm", b, p)
        for name in ("A", "B", "C"):
            assert rel(gs[name], rs[name]) < tol["F"], (name, b, rel(gs[name], rs[name]))
        f_ref = oracle.fit(X_fit[:k], rs["A"], rs["B"], rs["C"])
        assert abs(gs["fit"] - f_ref) < tol["fit"], ("fit", b, gs["fit"], f_ref)
        assert fms((gs["A"], gs["B"], gs["C"]), (rs["A"], rs["B"], rs["C"])) > tol["fms"]


CASES_FP32 = {
    # the small dense workload: 100^3, rank 5, 80 old slices + 20 new, P=4, Q=20, S=5
    "c1": Case(100, 100, 5, 4, 20, 5, 80, (20,), 50),
    # ragged shapes (partial 64/128 tiles, R padded 7 -> 8), two batches
    "ragged": Case(130, 70, 7, 3, 17, 4, 9, (9, 5), 20, seed=3),
    # Qd = 52 > I = 40 and > J = 50: full-column-rank lift for both modes
    "overdetermined": Case(40, 50, 4, 6, 12, 4, 20, (8,), 25, seed=4),
    # one new slice per batch, R = 1
    "single_slice_rank1": Case(30, 33, 1, 2, 6, 2, 10, (1, 1), 15, seed=5),
}


@pytest.mark.parametrize("name", sorted(CASES_FP32))
def test_update_parity_fp32(pkg, name):
    case = CASES_FP32[name]
    d = case.make()
    _, ref = case.oracle_run(d)
    g, gpu = run_gpu(pkg, case, d)
    g.close()
    check_update(case, d, gpu, ref)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_update_parity_reduced_precision(pkg, prec):
    case = Case(100, 100, 5, 4, 20, 5, 80, (20,), 50, prec=prec, seed=7)
    d = case.make()
    _, ref = case.oracle_run(d)
    g, gpu = run_gpu(pkg, case, d)
    g.close()
    check_update(case, d, gpu, ref)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_stateless_compression_parity(pkg, prec):
    I, J, P, Q, S, t = 150, 130, 3, 24, 4, 7
    case = Case(I, J, 4, P, Q, S, t, (), 1, prec=prec, seed=11)
    d = case.make()
    Z = pkg.compress(I, J, P, Q, S, slices(d["X"], prec), dev(d["U"]), dev(d["V"]),
                     dev(d["W"][0]), prec=prec)
    for p in range(P):
        ref = oracle.compress(d["X"], oracle.replica_block(d["U"], p, Q, S),
                              oracle.replica_block(d["V"], p, Q, S),
                              oracle.replica_block(d["W"][0], p, Q, S))
        assert rel(Z[p], ref) < TOL[prec]["Y"], (p, rel(Z[p], ref))


def test_host_inputs_give_the_device_result(pkg):
    """The end-to-end path (host buffers copied by the library) is bitwise the
    device path."""
    case = CASES_FP32["ragged"]
    d = case.make()
    g1, out1 = run_gpu(pkg, case, d, upto=1)
    g2 = pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters, case.prec)
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    g2.init(f32(d["X"][:case.t_old]), f32(d["U"]), f32(d["V"]), f32(d["W"][0]), f32(d["A0"]),
            f32(d["B0"]), f32(d["C0"]))
    t = case.batches[0]
    g2.append(f32(d["X"][case.t_old:case.t_old + t]), f32(d["W"][1]))
    A2, B2, C2 = g2.factors()
    assert np.array_equal(A2, out1[0]["A"]) and np.array_equal(B2, out1[0]["B"])
    assert np.array_equal(C2, out1[0]["C"])
    g1.close()
    g2.close()


def test_fit_of_given_factors(pkg):
    case = Case(64, 48, 3, 2, 8, 2, 12, (), 1, seed=9)
    d = case.make()
    g = pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, 1)
    g.init(dev(d["X"][:12]), dev(d["U"]), dev(d["V"]), dev(d["W"][0]), dev(d["A0"]),
           dev(d["B0"]), dev(d["C0"]))
    f = g.fit(dev(d["X"][:12]))
    g.close()
    assert abs(f - oracle.fit(d["X"][:12], d["A0"], d["B0"], d["C0"])) < 1e-6


def test_call_order_and_argument_errors(pkg):
    g = pkg.Octen(20, 20, 2, 2, 6, 2, 3)
    x = torch.zeros((2, 20, 20), device="cuda")
    w = torch.zeros((2, 10), device="cuda")
    with pytest.raises(pkg.OctenError) as e:
        g.append(x, w)
    assert e.value.status == 6          # ESTATE: append before init
    with pytest.raises(pkg.OctenError) as e:
        g.append_ptr(0, 1, 0)
    assert e.value.status in (1, 6)
    g.close()


def test_checkpoint_resume_is_bit_identical(pkg, tmp_path):
    """Save after one batch, load into a new context, append the next batch on
    both: identical summaries and factors."""
    case = CASES_FP32["ragged"]
    d = case.make()
    g = pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters, case.prec)
    g.init(slices(d["X"][:case.t_old], case.prec), dev(d["U"]), dev(d["V"]), dev(d["W"][0]),
           dev(d["A0"]), dev(d["B0"]), dev(d["C0"]))
    k = case.t_old
    t0, t1 = case.batches
    g.append(slices(d["X"][k:k + t0], case.prec), dev(d["W"][1]))
    path = str(tmp_path / "state.octen")
    g.save(path)
    h = pkg.Octen.load(path)
    xs = slices(d["X"][k + t0:k + t0 + t1], case.prec)
    g.append(xs, dev(d["W"][2]))
    h.append(xs, dev(d["W"][2]))
    for a, b in zip(g.factors(), h.factors()):
        assert np.array_equal(a, b)
    assert np.array_equal(g.replicas(), h.replicas())
    g.close()
    h.close()


def test_append_many_uneven_streams(pkg):
    """Several independent streams with uneven shapes, ranks and batch sizes,
    each on its own CUDA stream, appended in one octen_append_many call: each
    matches the oracle (bf16 tolerances) and equals its own single-stream
    octen_append bit for bit."""
    rng = np.random.default_rng(41)
    cases = []
    for i in range(4):
        R = int(rng.integers(2, 7))
        Q = int(rng.choice([12, 16, 20, 24]))
        S = min(R, Q // 2)
        cases.append(Case(int(rng.integers(40, 130)), int(rng.integers(40, 130)), R, 3, Q, S,
                          int(rng.integers(8, 20)), (int(rng.integers(3, 12)),), 20,
                          prec="bf16", seed=100 + i))
    datas = [c.make() for c in cases]
    streams = [torch.cuda.Stream() for _ in cases]

    def start(case, d, stream):
        g = pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters, case.prec,
                      stream=stream)
        g.init(slices(d["X"][:case.t_old], case.prec), dev(d["U"]), dev(d["V"]), dev(d["W"][0]),
               dev(d["A0"]), dev(d["B0"]), dev(d["C0"]))
        return g

    many = [start(c, d, s) for c, d, s in zip(cases, datas, streams)]
    torch.cuda.synchronize()
    xs = [slices(d["X"][c.t_old:c.t_old + c.batches[0]], c.prec) for c, d in zip(cases, datas)]
    ws = [dev(d["W"][1]) for d in datas]
    pkg.append_many(many, xs, ws)
    for c, d, g, x, w in zip(cases, datas, many, xs, ws):
        single = start(c, d, None)
        single.append(x, w)
        for a, b in zip(g.factors(), single.factors()):
            assert np.array_equal(a, b)
        _, ref = c.oracle_run(d)
        k = c.t_old + c.batches[0]
        A, B, C = g.factors()
        f = g.fit(slices(d["X"][:k], c.prec))
        f_ref = oracle.fit(d["X"][:k], ref[0]["A"], ref[0]["B"], ref[0]["C"])
        assert abs(f - f_ref) < TOL["bf16"]["fit"], (f, f_ref)
        assert fms((A, B, C), (ref[0]["A"], ref[0]["B"], ref[0]["C"])) > TOL["bf16"]["fms"]
        single.close()
        g.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_init_decomposition_matches_oracle(pkg, prec):
    """octen_init without C0: the existing decomposition is a CP-ALS of X_old
    on the GPU from the guesses A0, B0; it and the update that follows match
    the oracle doing the same (oracle.decompose_existing)."""
    case = Case(60, 50, 4, 3, 12, 3, 30, (10,), 30, prec=prec, seed=62)
    d = case.make()
    g = pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters, case.prec)
    g.init(slices(d["X"][:case.t_old], case.prec), dev(d["U"]), dev(d["V"]), dev(d["W"][0]),
           dev(d["A0"]), dev(d["B0"]), None)
    A, B, C = g.factors()
    Ar, Br, Cr = oracle.decompose_existing(d["X"][:case.t_old], d["A0"], d["B0"], case.iters)
    tol = TOL[prec]
    for name, x, y in (("A", A, Ar), ("B", B, Br), ("C", C, Cr)):
        assert rel(x, y) < tol["F"], (name, rel(x, y))
    f_gpu = g.fit(slices(d["X"][:case.t_old], case.prec))
    f_ref = oracle.fit(d["X"][:case.t_old], Ar, Br, Cr)
    assert abs(f_gpu - f_ref) < tol["fit"], (f_gpu, f_ref)
    assert f_ref > 0.98
    # the update from there
    o = oracle.OctenOracle(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters)
    o.init(d["X"][:case.t_old], d["U"], d["V"], d["W"][0], d["A0"], d["B0"], None)
    k = case.t_old
    g.append(slices(d["X"][k:k + 10], case.prec), dev(d["W"][1]))
    o.append(d["X"][k:k + 10], d["W"][1])
    A, B, C = g.factors()
    assert fms((A, B, C), (o.A, o.B, o.C)) > tol["fms"]
    assert abs(g.fit(slices(d["X"][:k + 10], case.prec))
               - oracle.fit(d["X"][:k + 10], o.A, o.B, o.C)) < tol["fit"]
    g.close()


def test_append_many_steps_as_one_graph_equal_single_appends(pkg):
    """Four octen_append_many steps over uneven streams (small replicas on the
    single-launch CP-ALS, Q = 40 on the tensor cores, Q = 36 zero-padded to 40):
    once every stream has a recorded tail (from the third step) a step is one
    graph launch, with each context's ALS GEMMs on a share of the SMs.  Every
    stream equals the same appends made one by one with octen_append, bit for
    bit, and its launches are counted."""
    cases = [Case(96, 80, 4, 3, 20, 4, 8, (6,) * 4, 6, prec="bf16", seed=130),
             Case(160, 144, 6, 3, 40, 6, 8, (8,) * 4, 6, prec="bf16", seed=131),
             Case(128, 112, 5, 2, 36, 5, 8, (5,) * 4, 6, prec="bf16", seed=132)]
    datas = [c.make() for c in cases]
    streams = [torch.cuda.Stream() for _ in cases]

    def start(case, d, stream):
        g = pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters, case.prec,
                      stream=stream)
        g.init(slices(d["X"][:case.t_old], case.prec), dev(d["U"]), dev(d["V"]), dev(d["W"][0]),
               dev(d["A0"]), dev(d["B0"]), dev(d["C0"]))
        return g

    def batch(c, d, b):
        k = c.t_old + sum(c.batches[:b])
        return slices(d["X"][k:k + c.batches[b]], c.prec), dev(d["W"][b + 1])

    many = [start(c, d, s) for c, d, s in zip(cases, datas, streams)]
    counts = []
    for b in range(4):
        xs, ws = zip(*[batch(c, d, b) for c, d in zip(cases, datas)])
        n0 = pkg.launch_count()
        pkg.append_many(many, list(xs), list(ws))
        counts.append(pkg.launch_count() - n0)
    # the graph steps run (and count) the same kernels as the eager ones
    assert counts[2] == counts[3] and counts[3] > 0
    for c, d, g in zip(cases, datas, many):
        single = start(c, d, None)
        for b in range(4):
            single.append(*batch(c, d, b))
        assert g.rows == single.rows == c.t_old + sum(c.batches)
        for a, s in zip(g.factors(), single.factors()):
            assert np.array_equal(a, s)
        assert np.array_equal(g.replicas(), single.replicas())
        single.close()
        g.close()
