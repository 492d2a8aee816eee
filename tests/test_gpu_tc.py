"""The tcgen05 tensor-core contractions (mode 2 and mode 1 of the compression)
against the FP64 oracle and against the independent SIMT kernels, on shapes
whose operand pitches satisfy the TMA rules (so the tensor-core path runs):
ragged M, N and K tails, several tiles in every dimension, Q not a multiple
of the 128-row tile."""
import os

import numpy as np
import pytest

import oracle
from tests._cases import Case, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_Y = {"bf16": 5e-3, "fp8": 6e-2}


@pytest.fixture(scope="module")
def pkg():
    import paper_1807_01350_gb300 as p

    assert torch.cuda.is_available()
    p.lib()
    return p


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a, np.float32), device="cuda").to(dtype)


SHAPES = [
    # I, J, P, Q, S, t
    (152, 144, 3, 24, 4, 7),
    (256, 512, 4, 80, 8, 5),
    (136, 208, 2, 200, 20, 3),
]


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("shape", SHAPES)
def test_tc_compression_matches_oracle_and_simt(pkg, prec, shape, monkeypatch):
    I, J, P, Q, S, t = shape
    case = Case(I, J, 4, P, Q, S, t, (), 1, prec=prec, seed=21)
    d = case.make()
    args = (I, J, P, Q, S, dev(d["X"], torch.bfloat16), dev(d["U"]), dev(d["V"]),
            dev(d["W"][0]))
    n0 = pkg.tc_launch_count()
    Z_tc = pkg.compress(*args, prec=prec)
    assert pkg.tc_launch_count() - n0 == 2, "both contractions should run on tcgen05"
    monkeypatch.setenv("OCTEN_GEMM", "simt")
    n1 = pkg.tc_launch_count()
    Z_simt = pkg.compress(*args, prec=prec)
    assert pkg.tc_launch_count() == n1
    for p in range(P):
        ref = oracle.compress(d["X"], oracle.replica_block(d["U"], p, Q, S),
                              oracle.replica_block(d["V"], p, Q, S),
                              oracle.replica_block(d["W"][0], p, Q, S))
        assert rel(Z_tc[p], ref) < TOL_Y[prec], (p, rel(Z_tc[p], ref))
        # same operands, same bf16 rounding of the intermediate; only the fp32
        # accumulation order differs
        assert rel(Z_tc[p], Z_simt[p]) < 2e-3, (p, rel(Z_tc[p], Z_simt[p]))


def test_tc_update_parity_bf16(pkg):
    """A whole update on the tensor-core path (J, I multiples of 16)."""
    from tests.test_gpu_parity import check_update, run_gpu

    case = Case(160, 144, 6, 4, 32, 8, 40, (16, 16), 30, prec="bf16", seed=22)
    d = case.make()
    _, ref = case.oracle_run(d)
    n0 = pkg.tc_launch_count()
    g, gpu = run_gpu(pkg, case, d)
    g.close()
    assert pkg.tc_launch_count() > n0
    check_update(case, d, gpu, ref)


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_als_graph_replay_equals_eager_launches(pkg, prec, monkeypatch):
    """The replica CP-ALS recorded as a CUDA graph at the first append and
    replayed afterwards gives the factors of the same kernels launched one by
    one (OCTEN_GRAPH=0) bit for bit, and its launches are still counted."""
    from tests.test_gpu_parity import run_gpu

    case = Case(160, 144, 6, 4, 32, 8, 40, (16, 8, 16), 12, prec=prec, seed=23)
    d = case.make()
    n0 = pkg.launch_count()
    g, graph = run_gpu(pkg, case, d)
    g.close()
    n_graph = pkg.launch_count() - n0
    monkeypatch.setenv("OCTEN_GRAPH", "0")
    n1 = pkg.launch_count()
    h, eager = run_gpu(pkg, case, d)
    h.close()
    assert pkg.launch_count() - n1 == n_graph
    for a, b in zip(graph, eager):
        for key in ("Y", "A", "B", "C"):
            assert np.array_equal(a[key], b[key]), key
        for u, v in zip(a["raw"], b["raw"]):
            assert np.array_equal(u, v)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_single_launch_small_replica_als(pkg, prec, monkeypatch):
    """Small replicas (Q = 20) run their whole CP-ALS in one launch; the result
    matches the oracle and the multi-launch path (OCTEN_ALS_FUSED=0), and an
    append issues far fewer launches."""
    from tests.test_gpu_parity import check_update, run_gpu

    case = Case(100, 100, 5, 4, 20, 5, 40, (20, 10), 50, prec=prec, seed=24)
    d = case.make()
    _, ref = case.oracle_run(d)
    n0 = pkg.launch_count()
    g, fused = run_gpu(pkg, case, d)
    g.close()
    n_fused = pkg.launch_count() - n0
    check_update(case, d, fused, ref)
    monkeypatch.setenv("OCTEN_ALS_FUSED", "0")
    n1 = pkg.launch_count()
    h, multi = run_gpu(pkg, case, d)
    h.close()
    n_multi = pkg.launch_count() - n1
    check_update(case, d, multi, ref)
    assert n_fused * 4 < n_multi, (n_fused, n_multi)
    for a, b in zip(fused, multi):
        for key in ("A", "B", "C"):
            assert np.allclose(a[key], b[key], rtol=1e-3, atol=1e-4), key


def test_autotuned_gemms_give_bit_identical_results(pkg, monkeypatch):
    """The GEMM autotuner only picks among configurations with identical
    results: an update with the defaults (OCTEN_AUTOTUNE=0, run first so the
    process-wide choices for these shapes are not yet made) equals the same
    update with the tuned choices bit for bit."""
    from tests.test_gpu_parity import run_gpu

    case = Case(176, 152, 6, 3, 40, 8, 24, (16, 8, 16), 10, prec="bf16", seed=25)
    d = case.make()
    monkeypatch.setenv("OCTEN_AUTOTUNE", "0")
    g, plain = run_gpu(pkg, case, d)
    g.close()
    monkeypatch.delenv("OCTEN_AUTOTUNE")
    h, tuned = run_gpu(pkg, case, d)
    h.close()
    for a, b in zip(plain, tuned):
        for key in ("Y", "A", "B", "C"):
            assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("prec", ["bf16", "fp8", "fp32"])
def test_host_batches_copied_in_pieces_equal_device_batches(pkg, prec):
    """Host slices of an append are copied in pieces whose mode-2 contraction
    starts as each piece arrives; the result equals the same update from
    device-resident slices bit for bit (each output keeps its summation order)."""
    from tests.test_gpu_parity import dev, slices

    case = Case(96, 80, 5, 3, 16, 4, 12, (16, 5, 2), 8, prec=prec, seed=27)
    d = case.make()

    def host(a):
        import torch
        t = torch.as_tensor(np.asarray(a, np.float32))
        return t if prec == "fp32" else t.to(torch.bfloat16)

    out = []
    for conv in (lambda a: slices(a, prec), host):
        g = pkg.Octen(case.I, case.J, case.R, case.P, case.Q, case.S, case.iters, prec)
        g.init(slices(d["X"][:case.t_old], prec), dev(d["U"]), dev(d["V"]), dev(d["W"][0]),
               dev(d["A0"]), dev(d["B0"]), dev(d["C0"]))
        k = case.t_old
        states = []
        for b, t in enumerate(case.batches):
            g.append(conv(d["X"][k:k + t]), np.asarray(d["W"][b + 1], np.float32))
            k += t
            A, B, C = g.factors()
            states.append((g.replicas(), A, B, C))
        g.close()
        out.append(states)
    for a, b in zip(*out):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("Q", [32, 40])
def test_replica_groups_give_bit_identical_results(pkg, Q, monkeypatch):
    """The tensor-core CP-ALS run as independent chains over groups of
    replicas (OCTEN_ALS_GROUPS, each group's GEMMs on a share of the SMs)
    gives the single chain's results bit for bit: per replica the launches
    and their summation order are the same.  Q = 40 takes the segmented
    partial sums (32 does not divide Q); three appends cover the eager first
    append and the graph replays."""
    from tests.test_gpu_parity import run_gpu

    case = Case(160, 144, 6, 5, Q, 8, 24, (16, 8, 16), 10, prec="bf16", seed=28)
    d = case.make()
    runs = {}
    for groups in ("1", "2", "3"):
        monkeypatch.setenv("OCTEN_ALS_GROUPS", groups)
        g, states = run_gpu(pkg, case, d)
        g.close()
        runs[groups] = states
    for groups in ("2", "3"):
        for a, b in zip(runs["1"], runs[groups]):
            for key in ("Y", "A", "B", "C"):
                assert np.array_equal(a[key], b[key]), (groups, key)
            for u, v in zip(a["raw"], b["raw"]):
                assert np.array_equal(u, v), groups


@pytest.mark.parametrize("Q", [36, 45])
def test_padded_replicas_run_the_tensor_core_als(pkg, Q, monkeypatch):
    """Q not a multiple of 8 (the bf16 row pitch the TMA loads need): the
    replica CP-ALS runs on tcgen05 with X_p zero-padded to the next multiple
    of 8, and the update matches the oracle at the bf16 tolerances and the
    SIMT path (OCTEN_GEMM=simt) closely."""
    from tests.test_gpu_parity import check_update, run_gpu

    case = Case(160, 144, 6, 3, Q, 6, 24, (16, 8), 10, prec="bf16", seed=29)
    d = case.make()
    _, ref = case.oracle_run(d)
    n0 = pkg.tc_launch_count()
    g, tc = run_gpu(pkg, case, d)
    g.close()
    # per append: mode 2, mode 1, and two GEMMs per sweep plus the final C update
    assert pkg.tc_launch_count() - n0 >= len(case.batches) * (2 + 2 * case.iters + 1)
    check_update(case, d, tc, ref)
    monkeypatch.setenv("OCTEN_GEMM", "simt")
    h, simt = run_gpu(pkg, case, d)
    h.close()
    for a, b in zip(tc, simt):
        assert abs(a["fit"] - b["fit"]) < 1e-3
        for key in ("A", "B", "C"):
            assert rel(a[key], b[key]) < 5e-2, key


def test_refused_tensor_core_launches_are_counted(pkg):
    """A bf16 compression whose operand rows meet the TMA pitch rule runs both
    contractions on tcgen05 with no fallback; one whose slice rows are 150
    bf16 (300 bytes, not a multiple of 16) runs mode 2 on the SIMT kernels,
    and that refused launch is counted (the first of a process is also
    reported on stderr); the result is right either way."""
    for (I, J), want_fallback in (((152, 144), False), ((152, 150), True)):
        P, Q, S, t = 3, 24, 4, 5
        case = Case(I, J, 4, P, Q, S, t, (), 1, prec="bf16", seed=26)
        d = case.make()
        f0 = pkg.tc_fallback_count()
        Z = pkg.compress(I, J, P, Q, S, dev(d["X"], torch.bfloat16), dev(d["U"]), dev(d["V"]),
                         dev(d["W"][0]), prec="bf16")
        assert (pkg.tc_fallback_count() > f0) == want_fallback, (J, pkg.tc_fallback_count(), f0)
        for p in range(P):
            ref = oracle.compress(d["X"], oracle.replica_block(d["U"], p, Q, S),
                                  oracle.replica_block(d["V"], p, Q, S),
                                  oracle.replica_block(d["W"][0], p, Q, S))
            assert rel(Z[p], ref) < TOL_Y["bf16"]
