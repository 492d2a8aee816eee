"""GPU parity of the N-mode extension (Sec. "Extending to Higher-Order
Tensors"): the CUDA path through the octen_n_* C ABI against the FP64 N-mode
oracle on the same seeded inputs, stage by stage (summaries, raw replica CP,
matching permutation, lifted factors, fit), for N = 3 .. 6 modes.

Tolerances are the fp32 ones of the 3-mode update: summaries within 1e-5
relative Frobenius error per replica (fp32 FFMA accumulation), replica and
lifted factors within 1e-3 (fp32 lift operators and fp32 ALS substitutions),
identical matching permutations, fit within 1e-4 and a factor-match score
against the oracle's factors above 0.999."""
import numpy as np
import pytest

from oracle import octen_n
from tests._cases import rel
from tests._metrics import fms
from tests._ncases import NCase

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = dict(Y=1e-5, F=1e-3, fit=1e-4, fms=0.999)

CASES = {
    # three modes through the N-mode path (equals the 3-mode update in fp32)
    "n3": NCase((40, 30), 4, 3, 8, 3, 12, (5, 3), 30, seed=11),
    # four modes, several GEMM tiles and ragged tails, two batches
    "n4": NCase((40, 36, 30), 4, 4, 8, 3, 10, (10, 4), 40, seed=12),
    # Qd = 22 above every I_n: full-column-rank lift in every mode; R = 5 padded to 8
    "n4_overdetermined": NCase((9, 11, 7), 5, 4, 7, 2, 12, (1, 2), 30, seed=13),
    # five and six modes
    "n5": NCase((7, 6, 8, 5), 3, 3, 5, 2, 8, (3,), 30, seed=14),
    "n6": NCase((5, 4, 6, 3, 4), 2, 2, 4, 1, 6, (2,), 25, seed=15),
    # R = 1, one slice per batch
    "n4_rank1_single": NCase((12, 10, 9), 1, 2, 5, 2, 6, (1, 1), 20, seed=16),
    # slices large enough that one compression pass takes fewer slices than
    # the existing tensor holds (two passes at init)
    "n4_chunked": NCase((300, 300, 4), 2, 2, 4, 2, 50, (5,), 20, seed=17),
    # summaries too large for shared memory (read from global memory) and an
    # outer index table too large for the Khatri-Rao form (the odometer MTTKRP):
    # six modes with Q = 8, and three modes with Q = 40 > 32
    "n6_global": NCase((6, 5, 4, 5, 6), 2, 2, 8, 2, 6, (2,), 10, seed=18),
    "n3_q40": NCase((48, 44), 3, 2, 40, 4, 8, (3,), 10, seed=19),
}


@pytest.fixture(scope="module")
def pkg():
    import paper_1807_01350_gb300 as p

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    p.lib()
    return p


def dev(a):
    return torch.as_tensor(np.asarray(a, np.float32), device="cuda")


def run_gpu(pkg, case, d, host=False):
    g = pkg.OctenN(case.dims, case.R, case.P, case.Q, case.S, case.iters)
    conv = (lambda a: np.asarray(a, np.float32)) if host else dev
    g.init(conv(d["X"][:case.t_old]), [conv(u) for u in d["U"]], conv(d["W"][0]),
           [conv(a) for a in d["A0"]], conv(d["C0"]))
    k = case.t_old
    out = []
    for b, t in enumerate(case.batches):
        g.append(conv(d["X"][k:k + t]), conv(d["W"][b + 1]))
        k += t
        As, C = g.factors()
        out.append(dict(Y=g.replicas(), A=As, C=C, raw=g.replica_factors(0),
                        hat=g.replica_factors(1), fit=g.fit(conv(d["X"][:k]))))
    return g, out


def check(case, d, gpu, ref):
    k = case.t_old
    for b, (gs, rs) in enumerate(zip(gpu, ref)):
        k += case.batches[b]
        for p in range(case.P):
            e = rel(gs["Y"][p], rs["Y"][p])
            assert e < TOL["Y"], ("Y", b, p, e)
        Fs, perm, scales = gs["raw"]
        for p in range(case.P):
            for n in range(case.N):
                e = rel(Fs[n][p], rs["raw"][p][n])
                assert e < TOL["F"], ("raw", b, p, n, e)
        Fh, perm, scales = gs["hat"]
        for p in range(case.P):
            assert np.array_equal(perm[p], rs["hat"][p][2]), ("perm", b, p)
            for n in range(case.N - 1):
                e = rel(Fh[n][p], rs["hat"][p][0][n])
                assert e < TOL["F"], ("hat", b, p, n, e)
            e = rel(Fh[case.N - 1][p], rs["hat"][p][1])
            assert e < TOL["F"], ("hat C", b, p, e)
        for n in range(case.N - 1):
            e = rel(gs["A"][n], rs["A"][n])
            assert e < TOL["F"], ("A", b, n, e)
        assert rel(gs["C"], rs["C"]) < TOL["F"], ("C", b, rel(gs["C"], rs["C"]))
        f_gpu = octen_n.fit_n(d["X"][:k], [np.asarray(a, np.float64) for a in gs["A"]],
                              np.asarray(gs["C"], np.float64))
        f_ref = octen_n.fit_n(d["X"][:k], rs["A"], rs["C"])
        assert abs(f_gpu - f_ref) < TOL["fit"], ("fit", b, f_gpu, f_ref)
        # the library's own fit of its factors (octen_n_fit, fp64 sums)
        assert abs(gs["fit"] - f_gpu) < 1e-9, ("octen_n_fit", b, gs["fit"], f_gpu)
        assert fms(tuple(gs["A"]) + (gs["C"],), tuple(rs["A"]) + (rs["C"],)) > TOL["fms"]


@pytest.mark.parametrize("name", sorted(CASES))
def test_nmode_update_parity(pkg, name):
    case = CASES[name]
    d = case.make()
    _, ref = case.oracle_run(d)
    g, gpu = run_gpu(pkg, case, d)
    g.close()
    check(case, d, gpu, ref)


def test_nmode_host_inputs_match_device_inputs(pkg):
    case = CASES["n4"]
    d = case.make()
    g1, a = run_gpu(pkg, case, d, host=False)
    g2, b = run_gpu(pkg, case, d, host=True)
    g1.close()
    g2.close()
    for x, y in zip(a, b):
        assert np.array_equal(x["Y"], y["Y"])
        assert np.array_equal(x["C"], y["C"])
        for u, v in zip(x["A"], y["A"]):
            assert np.array_equal(u, v)


def test_nmode_rejects_bad_shapes(pkg):
    with pytest.raises(pkg.OctenError):
        pkg.OctenN((10, 10, 10, 10, 10, 10), 2, 2, 4, 1, 5)    # N = 7
    with pytest.raises(pkg.OctenError):
        pkg.OctenN((10, 10), 2, 2, 4, 4, 5)                     # S = Q
    g = pkg.OctenN((6, 5, 4), 2, 2, 4, 1, 5)
    with pytest.raises(pkg.OctenError):
        g.append(np.zeros((1, 6, 5, 4), np.float32), np.zeros((1, 7), np.float32))  # before init
    g.close()


def test_nmode_checkpoint_resume_is_bit_identical(pkg, tmp_path):
    """octen_n_save after an update and octen_n_load into a fresh context: the
    next update gives the same factors and summaries, bit for bit, as the
    context that was saved."""
    case = CASES["n4"]
    d = case.make()
    g = pkg.OctenN(case.dims, case.R, case.P, case.Q, case.S, case.iters)
    g.init(dev(d["X"][:case.t_old]), [dev(u) for u in d["U"]], dev(d["W"][0]),
           [dev(a) for a in d["A0"]], dev(d["C0"]))
    k = case.t_old
    t0, t1 = case.batches[:2]
    g.append(dev(d["X"][k:k + t0]), dev(d["W"][1]))
    path = str(tmp_path / "nmode.ckpt")
    g.save(path)
    X1, W1 = dev(d["X"][k + t0:k + t0 + t1]), dev(d["W"][2])
    g.append(X1, W1)
    A_a, C_a = g.factors()
    Y_a = g.replicas()
    g.close()
    h = pkg.OctenN.load(path)
    assert h.dims == list(case.dims) and h.rows == k + t0
    h.append(X1, W1)
    A_b, C_b = h.factors()
    Y_b = h.replicas()
    h.close()
    assert np.array_equal(C_a, C_b) and np.array_equal(Y_a, Y_b)
    for a, b in zip(A_a, A_b):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["n3", "n4", "n5"])
def test_nmode_init_decomposition_matches_oracle(pkg, name):
    """octen_n_init without C0: the existing decomposition is the N-way CP-ALS
    of X_old on the GPU (one pass over X_old per mode per sweep) from the
    guesses A0; it and the update that follows match the oracle doing the same
    (octen_n.decompose_existing_n), at the fp32 tolerances."""
    case = CASES[name]
    d = case.make()
    X_old = d["X"][:case.t_old]
    g = pkg.OctenN(case.dims, case.R, case.P, case.Q, case.S, case.iters)
    g.init(dev(X_old), [dev(u) for u in d["U"]], dev(d["W"][0]), [dev(a) for a in d["A0"]],
           None)
    As, C = g.factors()
    ref = octen_n.decompose_existing_n(X_old, d["A0"], case.iters)
    for n in range(case.N - 1):
        assert rel(As[n], ref[n]) < TOL["F"], (n, rel(As[n], ref[n]))
    assert rel(C, ref[-1]) < TOL["F"], rel(C, ref[-1])
    f_gpu = octen_n.fit_n(X_old, [np.asarray(a, np.float64) for a in As],
                          np.asarray(C, np.float64))
    f_ref = octen_n.fit_n(X_old, ref[:-1], ref[-1])
    assert abs(f_gpu - f_ref) < TOL["fit"], (f_gpu, f_ref)
    assert f_ref > 0.98
    # the update from there
    o = octen_n.OctenOracleN(list(case.dims), case.R, case.P, case.Q, case.S, case.iters)
    o.init(X_old, d["U"], d["W"][0], d["A0"], None)
    k, t = case.t_old, case.batches[0]
    o.append(d["X"][k:k + t], d["W"][1])
    g.append(dev(d["X"][k:k + t]), dev(d["W"][1]))
    As, C = g.factors()
    g.close()
    for n in range(case.N - 1):
        assert rel(As[n], o.A[n]) < TOL["F"], (n, rel(As[n], o.A[n]))
    assert rel(C, o.C) < TOL["F"]
    assert fms(tuple(As) + (C,), tuple(o.A) + (o.C,)) > TOL["fms"]


def _bf16_case(case):
    """The case's inputs with the slices and every projection rounded to bf16
    (what a bf16 context receives and keeps)."""
    from synth import round_to

    d = case.make()
    d["X"] = round_to(d["X"], "bf16")
    d["U"] = [round_to(u, "bf16") for u in d["U"]]
    return d


def _bf16(a):
    return dev(a).to(torch.bfloat16)


@pytest.mark.parametrize("dims", [(40, 36, 32), (30, 28, 21)])
def test_nmode_bf16_update_parity(pkg, dims):
    """bf16 slices (N = 4): the slice-reading first contraction of the
    compression runs in bf16 with fp32 accumulation, on tcgen05 when the
    innermost size is a multiple of 8 (32) and on the SIMT kernels otherwise
    (21).  bf16 products are exact in fp32, so against the oracle run on the
    same bf16-rounded slices and projections the fp32 tolerances hold."""
    case = NCase(dims, 4, 4, 8, 3, 10, (10, 4), 40, seed=22)
    d = _bf16_case(case)
    _, ref = case.oracle_run(d)
    n_tc = pkg.tc_launch_count()
    g = pkg.OctenN(case.dims, case.R, case.P, case.Q, case.S, case.iters, prec="bf16")
    g.init(_bf16(d["X"][:case.t_old]), [dev(u) for u in d["U"]], dev(d["W"][0]),
           [dev(a) for a in d["A0"]], dev(d["C0"]))
    k = case.t_old
    gpu = []
    for b, t in enumerate(case.batches):
        g.append(_bf16(d["X"][k:k + t]), dev(d["W"][b + 1]))
        k += t
        As, C = g.factors()
        gpu.append(dict(Y=g.replicas(), A=As, C=C, raw=g.replica_factors(0),
                        hat=g.replica_factors(1), fit=g.fit(_bf16(d["X"][:k]))))
    g.close()
    if dims[-1] % 8 == 0:
        assert pkg.tc_launch_count() > n_tc, "the first contraction should run on tcgen05"
    check(case, d, gpu, ref)


def test_nmode_bf16_init_decomposition_matches_oracle(pkg):
    """A bf16 context initialised without C0: the N-way CP-ALS of the bf16
    slices matches the oracle's decomposition of the same values."""
    case = CASES["n4"]
    d = _bf16_case(case)
    X_old = d["X"][:case.t_old]
    g = pkg.OctenN(case.dims, case.R, case.P, case.Q, case.S, case.iters, prec="bf16")
    g.init(_bf16(X_old), [dev(u) for u in d["U"]], dev(d["W"][0]), [dev(a) for a in d["A0"]],
           None)
    As, C = g.factors()
    g.close()
    ref = octen_n.decompose_existing_n(X_old, d["A0"], case.iters)
    for n in range(case.N - 1):
        assert rel(As[n], ref[n]) < TOL["F"], (n, rel(As[n], ref[n]))
    assert rel(C, ref[-1]) < TOL["F"]
