"""Host-side accounting of the benchmark (no GPU): algorithmic work per launch,
the roofline entry built from it, the whole-job rate and the clock record.

The per-launch byte counts of the replica CP-ALS GEMMs are checked against the
buffer sizes of the 4000^2 stream (P = 16 replicas of 256^3, R = 32, 30
sweeps): the bf16 copy of X_p (Q^3 per replica), the bf16 transposed factor
(32 rows of Q), the fp32 partial sums over 32 consecutive rows and the bf16 Tc
(Q^2 rows of 32), as the tensor-core profile of these GEMMs lists them.
"""
import os
import tempfile

import pytest

import bench
from synth import WORKLOADS

MB = 1e6


def test_stage_work_of_the_4000_squared_stream():
    wl = WORKLOADS["c4"]
    assert (wl.I, wl.J, wl.batch, wl.P, wl.Q, wl.R, wl.Qd) == (4000, 4000, 16, 16, 256, 32, 3616)
    w = bench.stage_work(wl, "bf16", layouts=True)
    # mode 2: a (16 * 4000) x 4000 by 4000 x 3616 product
    assert w["mode2"][0] == pytest.approx(2 * 16 * 4000 * 4000 * 3616)
    # mode 3: Y_p read and written in fp32, T2 read in fp32, two bf16 copies written
    y = 16 * 256 ** 3 * 4
    assert w["mode3"][1] == pytest.approx(2 * y + 16 * 16 * 256 * 256 * 4 + 2 * 16 * 256 ** 3 * 2)
    assert w["mode3"][1] == pytest.approx(3.29e9, rel=0.01)
    no_copies = bench.stage_work(wl, "bf16", layouts=False)["mode3"][1]
    assert w["mode3"][1] - no_copies == pytest.approx(2 * 16 * 256 ** 3 * 2)


def test_als_gemm_bytes_match_the_profiled_buffers():
    wl = WORKLOADS["c4"]
    x_copy = 16 * 256 ** 3 * 2                 # 536.9 MB
    factor_t = 16 * 32 * 256 * 2               # 0.26 MB
    partials = 16 * 256 * (256 // 32) * 32 * 4  # 4.2 MB
    tc_out = 16 * 256 * 256 * 32 * 2           # 67.1 MB
    m3 = x_copy + factor_t + partials
    tc = x_copy + factor_t + tc_out + partials
    assert m3 / MB == pytest.approx(541.3, abs=0.1)
    assert tc / MB == pytest.approx(608.4, abs=0.1)
    # 31 M3 launches (one per sweep and the final C update) and 30 Tc launches
    assert bench.als_gemm_tc_bytes(wl) == pytest.approx((31 * m3 + 30 * tc) / 61)


def test_als_gemm_bytes_when_32_does_not_divide_q():
    # Q = 200: every block of 32 rows writes two segment sums
    wl = WORKLOADS["c3"]
    assert wl.Q % 32 != 0 and wl.Q >= 32
    P, Q, it = wl.P, wl.Q, wl.als_iters
    RT = 32 if wl.R > 16 else (16 if wl.R > 8 else 8)
    blocks = -(-Q * Q // 32)
    partials = 2 * blocks * RT * 4 * P
    x_copy = 2 * P * Q ** 3
    factor_t = 2 * P * 32 * Q
    m3 = x_copy + factor_t + partials
    tc = m3 + 2 * P * Q * Q * RT
    assert bench.als_gemm_tc_bytes(wl) == pytest.approx(((it + 1) * m3 + it * tc) / (2 * it + 1))


def test_roofline_entry_is_consistent():
    wl = WORKLOADS["c4"]
    pk = dict(hbm=6787.0, bf16=2000.0, bf16_sus=1800.0, src="measured")
    r = bench.roofline_for("als_gemm", 0.0915, wl, "bf16", pk, 544.7e6, tc_stages=("als_gemm",))
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6787.0
    assert r["achieved"] == pytest.approx(bench.als_gemm_tc_bytes(wl) / 0.0915e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    assert r["traffic"] == 544.7e6
    # mode 2 on the tensor cores: fp8 doubles the bf16 peak
    r8 = bench.roofline_for("mode2", 1.0, wl, "fp8", pk, None, tc_stages=("mode2",))
    rb = bench.roofline_for("mode2", 1.0, wl, "bf16", pk, None, tc_stages=("mode2",))
    assert r8["bound"] == rb["bound"] == "tensor"
    assert r8["peak"] == pytest.approx(2 * rb["peak"])
    # the fp32 path is bound by the fp32 lanes
    r32 = bench.roofline_for("als_gemm", 1.0, wl, "fp32", pk, None)
    assert r32["bound"] == "alu"
    assert r32["peak"] == pytest.approx(152 * 128 * 2 * 2.070e-3, rel=1e-3)


def test_whole_job_rate_and_rank_seeds():
    # two ranks of 160 slices each, the slower taking 0.2 s
    assert bench.whole_job_rate(160, 0.2, 2) == pytest.approx(1600.0)
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    seeds = {bench.rank_seed(7, r) for r in range(8)}
    assert len(seeds) == 8


def test_clock_record_reads_reasons_and_median():
    rows = [
        "0, 1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1990, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(rows) + "\n")
    try:
        cs = bench.ClockSampler(0)
        cs.path = path
        s = cs.summary()
    finally:
        os.remove(path)
    assert s["sm_mhz"] == 1980.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3 and s["power_w_max"] == pytest.approx(1200.5)


def test_clock_record_without_samples_says_so():
    fd, path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    try:
        cs = bench.ClockSampler(0)
        cs.path = path
        s = cs.summary()
    finally:
        os.remove(path)
    assert s["reasons"] == ["unsampled"] and s["sm_mhz"] is None


def test_mode3_is_charged_the_method_bytes_with_the_copies_beside():
    wl = WORKLOADS["c4"]
    pk = dict(hbm=6690.8, bf16=1892.4, bf16_sus=1718.1, src="measured")
    tcs = ("mode2", "mode1", "als_gemm")
    r = bench.roofline_for("mode3", 0.69, wl, "bf16", pk, None, tc_stages=tcs)
    y = 16 * 256 ** 3 * 4
    t2 = 16 * 16 * 256 * 256 * 4
    # the scope table's bytes of the summary update: Y read and written, T2 read
    assert r["achieved"] == pytest.approx((2 * y + t2) / 0.69e-3 / 1e9, rel=1e-3)
    assert (2 * y + t2) / 1e9 == pytest.approx(2.22, abs=0.01)
    assert r["copy_bytes"] == 2 * 16 * 256 ** 3 * 2
    assert r["frac_incl_copies"] > r["frac"]
    # without the tensor-core ALS there are no copies to report
    r32 = bench.roofline_for("mode3", 0.69, wl, "fp32", pk, None, tc_stages=())
    assert "copy_bytes" not in r32


def test_compression_roofline_of_the_4000_squared_batch():
    wl = WORKLOADS["c4"]
    pk = dict(hbm=6690.8, bf16=1942.7, bf16_sus=1714.2, src="measured")
    tcs = ("mode2", "mode1", "als_gemm")
    comp = {s: {"ms_per_launch": ms} for s, ms in (("mode2", 1.27), ("mode1", 0.19),
                                                    ("mode3", 0.69))}
    c = bench.compression_at_roofline(wl, "bf16", pk, comp, tcs)
    # flops per slice 2 I J Qd + 2 P Q^2 I + 2 P Q^3 = 1.25e11, 16 slices at the
    # burst bf16 peak: the scope table's 1027 us per batch
    assert c["flops_per_batch"] / 16 == pytest.approx(1.246e11, rel=1e-3)
    assert c["flops_only_at_burst_peak_ms"] == pytest.approx(1.027, abs=0.002)
    # per stage the slower bound: mode 2 at the sustained tensor peak; mode 1
    # reads its 557 MB of mode-2 output slightly slower than it multiplies;
    # mode 3 at the HBM bandwidth for its 2.22 GB
    w = bench.stage_work(wl, "bf16")
    assert w["mode1"][1] / 6690.8e9 > w["mode1"][0] / 1714.2e12
    want = 1e3 * (w["mode2"][0] / 1714.2e12 + w["mode1"][1] / 6690.8e9 +
                  w["mode3"][1] / 6690.8e9)
    assert c["at_roofline_ms"] == pytest.approx(want, rel=1e-3)
    assert c["measured_ms"] == pytest.approx(2.15)
    assert c["frac"] == pytest.approx(want / 2.15, rel=1e-3)


def test_tensor_core_stages_report_their_binding_bound():
    """A tensor-core stage is reported against whichever of its two limits
    binds: mode 2 at 4000^2 by its flops (1.85 TFLOP against 1.07 GB), mode 1
    by its bytes (0.134 TFLOP against 557 MB: the mode-2 product it streams),
    each with the other fraction beside it."""
    wl = WORKLOADS["c4"]
    pk = {"hbm": 6690.8, "bf16": 1892.4, "bf16_sus": 1718.1, "src": "measured"}
    m2 = bench.roofline_for("mode2", 1.26, wl, "bf16", pk, None, ("mode2", "mode1"))
    m1 = bench.roofline_for("mode1", 0.18, wl, "bf16", pk, None, ("mode2", "mode1"))
    assert m2["bound"] == "tensor" and "hbm_frac" in m2
    assert m1["bound"] == "hbm" and "tensor_frac" in m1
    fl, nb = bench.stage_work(wl, "bf16")["mode1"]
    assert m1["achieved"] == pytest.approx(nb / 0.18e-3 / 1e9, rel=1e-3)
    assert m1["tensor_frac"] == pytest.approx(fl / 0.18e-3 / 1e12 / 1718.1, rel=1e-3)


def test_traffic_is_only_reported_for_the_captured_shape():
    """The ncu traffic figure belongs to the shape it was captured on: the
    4000^2 ALS GEMM has one, other workloads and precisions report none."""
    c4 = WORKLOADS["c4"].name
    assert bench.traffic_from_profiles("als_gemm", "bf16", c4) > 0
    assert bench.traffic_from_profiles("als_gemm", "bf16", WORKLOADS["c3"].name) is None
    assert bench.traffic_from_profiles("als_gemm", "fp8", c4) is None
    assert bench.traffic_from_profiles("mode2", "bf16", c4) is None
