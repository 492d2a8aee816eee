#!/usr/bin/env python3
"""Throughput of the OCTen online CP update on GB300: new slices per second.

One step = one `octen_append` of a batch of new slices (compression into the
P replicas, CP-ALS of every replica, anchor match, lift of A, B and the new
rows of C), with the batch already resident in HBM.  The default workload is
the 4000 x 4000-slice stream (rank 32, P = 16 replicas of 256^3, anchors
S = 32, batches of 16 slices, 64 existing slices, 30 CP-ALS sweeps); the
headline precision is bf16 (the precision whose fit stays within 1e-3 of the
FP64 oracle), with fp32 and fp8 runs of the same stream reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own independent stream (weak scaling, no
collective on the data path); the timed region is bracketed by barriers and
the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import contextlib
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from synth import WORKLOADS, factors, init_factors, projections, slice_batch  # noqa: E402
from synth import round_to, slice_batch_torch, time_projection, uneven_streams  # noqa: E402

METRIC = "new slices/sec (compress+CP update) at fit >= oracle-1e-3; BF16/FP8 vs FP32"
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12     # SMs x FP32 lanes x FMA x max clock


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return dict(hbm=float(d["hbm_gbs"]), bf16=float(d["bf16_tflops"]),
                    bf16_sus=float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                    src="measured")
    except Exception:
        return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, src="fallback")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        # the timed region starts once the sampler is producing samples
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < 5.0:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                pass
            time.sleep(0.02)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# ---------------------------------------------------------------------------
# one stream on the GPU
# ---------------------------------------------------------------------------
def stream_inputs(wl, prec, seed, nbatch, device):
    import torch

    K = wl.t_old + nbatch * wl.batch
    A, B, C = factors(wl.I, wl.J, K, wl.R, seed, cond=wl.cond, big_frac=wl.big_frac)
    U, V = projections(wl.I, wl.J, wl.P, wl.Q, wl.S, seed, prec)
    W = [time_projection(wl.t_old, wl.P, wl.Q, wl.S, seed, -1)]
    W += [time_projection(wl.batch, wl.P, wl.Q, wl.S, seed, b) for b in range(nbatch)]
    A0, B0, C0 = init_factors(A, B, C[:wl.t_old], 0.01, seed)
    dt = torch.float32 if prec == "fp32" else torch.bfloat16
    X = slice_batch_torch(A, B, C, 0, K, wl.noise, seed, device, dt)   # K x I x J in HBM
    f32 = lambda a: torch.as_tensor(np.asarray(a, np.float32), device=device)
    return dict(X=X, U=f32(U), V=f32(V), W=[f32(w) for w in W], A0=f32(A0), B0=f32(B0),
                C0=f32(C0))


def stage_work(wl, prec, layouts=False):
    """Algorithmic work per launch of each timed stage: (flops, bytes).  With
    `layouts` the mode-3 pass also writes the two bf16 copies of X_p that the
    tensor-core CP-ALS reads."""
    t, I, J, P, Q, R, Qd = wl.batch, wl.I, wl.J, wl.P, wl.Q, wl.R, wl.Qd
    xb = 4 if prec == "fp32" else (1 if prec == "fp8" else 2)
    return {
        "mode2": (2.0 * t * I * J * Qd, t * I * J * xb + Qd * J * xb + t * I * P * Q * (4 if prec == "fp32" else 2)),
        "mode1": (2.0 * t * P * Q * Q * I, t * P * Q * I * (4 if prec == "fp32" else 2) + P * Q * I * (4 if prec == "fp32" else 2)),
        "mode3": (2.0 * t * P * Q ** 3, 2.0 * 4 * P * Q ** 3 + 4.0 * t * P * Q * Q
                  + (2.0 * 2 * P * Q ** 3 if layouts else 0.0)),
        "als_gemm": (2.0 * P * Q ** 3 * R, 4.0 * P * Q ** 3),
        # e4m3 quantisation: an absmax pass and a scale-and-convert pass over the bf16 slices
        "quantize": (0.0, t * I * J * (2.0 + 2.0 + 1.0)),
    }


def als_gemm_tc_bytes(wl):
    """Algorithmic bytes per tensor-core ALS GEMM launch, averaged over an
    append (als_iters + 1 M3 launches, als_iters Tc launches).  The Tc GEMM
    reads the bf16 copy Xa and the bf16 C^T and writes Tc (bf16, rank padded
    to RT).  With Q >= 32 both GEMMs also write their fused partial sums over
    32 consecutive rows (fp32, RT per block; two segment sums per block when
    32 does not divide Q) and the M3 GEMM reads the bf16 copy Xc and the bf16
    B^T.  Below Q = 32 the M3 GEMM reads Xc and the Khatri-Rao operand (rank
    padded to 32), and the M1 reduction runs as a separate pass."""
    P, Q, R, it = wl.P, wl.Q, wl.R, wl.als_iters
    RT = 8 if R <= 8 else (16 if R <= 16 else 32)
    NP = 32
    QQ = Q * Q
    if Q >= 32:
        blocks = QQ // 32 if Q % 32 == 0 else 2 * ((QQ + 31) // 32)
        parts = 4.0 * P * blocks * RT
        m3 = 2.0 * P * Q ** 3 + 2.0 * P * NP * Q + parts
        tc = 2.0 * P * Q ** 3 + 2.0 * P * NP * Q + 2.0 * P * QQ * RT + parts
    else:
        m3 = 2.0 * P * Q ** 3 + 2.0 * P * NP * QQ
        tc = 2.0 * P * Q ** 3 + 2.0 * P * NP * Q + 2.0 * P * QQ * RT
    return ((it + 1) * m3 + it * tc) / (2 * it + 1)


def roofline_for(stage, ms_per_launch, wl, prec, pk, traffic, tc_stages=()):
    """Roofline entry of one stage.  Mode 3 is charged the method's bytes only
    (Y read and written, T2 read); when the tensor-core CP-ALS runs, the same
    pass also writes the two bf16 copies of X_p that the ALS reads, reported
    beside it as `copy_bytes` (they are the ALS's input, not the summary
    update's)."""
    flops, nbytes = stage_work(wl, prec)[stage]
    sec = ms_per_launch / 1e3
    extra = {}
    if stage == "mode3" and "als_gemm" in tc_stages:
        with_copies = stage_work(wl, prec, layouts=True)["mode3"][1]
        extra = {"copy_bytes": with_copies - nbytes,
                 "achieved_incl_copies": round(with_copies / sec / 1e9, 3),
                 "frac_incl_copies": round(with_copies / sec / 1e9 / pk["hbm"], 4)}
    if stage in ("mode3", "quantize"):
        bound, peak, unit, achieved = "hbm", pk["hbm"], "GB/s", nbytes / sec / 1e9
    elif stage == "als_gemm" and stage in tc_stages:
        bound, peak, unit = "hbm", pk["hbm"], "GB/s"
        achieved = als_gemm_tc_bytes(wl) / sec / 1e9
    elif stage in tc_stages:
        # the binding one of the two: flops at the sustained tensor peak or
        # the method's bytes at the copy bandwidth (mode 1 streams the 524 MB
        # mode-2 product at 4000^2 and is bound by its bytes)
        tpk = pk["bf16_sus"] * (2.0 if prec == "fp8" and stage == "mode2" else 1.0)
        t_flops, t_bytes = flops / (tpk * 1e12), nbytes / (pk["hbm"] * 1e9)
        if t_flops >= t_bytes:
            bound, peak, unit, achieved = "tensor", tpk, "TFLOP/s", flops / sec / 1e12
            extra["hbm_frac"] = round(nbytes / sec / 1e9 / pk["hbm"], 4)
        else:
            bound, peak, unit, achieved = "hbm", pk["hbm"], "GB/s", nbytes / sec / 1e9
            extra["tensor_frac"] = round(flops / sec / 1e12 / tpk, 4)
    else:
        bound, peak, unit, achieved = "alu", FP32_ALU_TFLOPS, "TFLOP/s", flops / sec / 1e12
    return dict({"kernel": stage, "bound": bound, "achieved": round(achieved, 3),
                 "peak": round(peak, 1), "unit": unit, "frac": round(achieved / peak, 4),
                 "traffic": traffic,
                 "peak_source": pk["src"] if bound != "alu" else
                 "derived: 152 SMs x 128 fp32 lanes x 2 flop x 2070 MHz",
                 "ms_per_launch": round(ms_per_launch, 4)}, **extra)


def compression_at_roofline(wl, prec, pk, comp, tc_stages):
    """The compression stages (quantise, mode 2, mode 1, mode 3) against their
    rooflines: each stage's time at the slower of its compute peak and the
    HBM bandwidth for the method's bytes, summed, over the measured sum; and
    the flops-only time at the burst tensor peak (the figure of the scope
    table: 2 t I J Qd + 2 t P Q^2 I + 2 t P Q^3 flop per batch)."""
    work = stage_work(wl, prec)
    stages = [s for s in ("quantize", "mode2", "mode1", "mode3") if s in comp]
    meas = sum(comp[s]["ms_per_launch"] for s in stages)
    roof = 0.0
    for s in stages:
        fl, nb = work[s]
        if s in tc_stages:
            cpk = pk["bf16_sus"] * (2.0 if prec == "fp8" and s == "mode2" else 1.0) * 1e12
        else:
            cpk = FP32_ALU_TFLOPS * 1e12
        roof += 1e3 * max(fl / cpk, nb / (pk["hbm"] * 1e9))
    tc = any(s in tc_stages for s in ("mode2", "mode1"))
    peak_b = (pk["bf16"] * (2.0 if prec == "fp8" else 1.0) if tc else FP32_ALU_TFLOPS) * 1e12
    fl_all = sum(work[s][0] for s in ("mode2", "mode1", "mode3"))
    return {"stages": stages, "measured_ms": round(meas, 4), "at_roofline_ms": round(roof, 4),
            "frac": round(roof / meas, 4) if meas > 0 else None,
            "flops_per_batch": fl_all,
            "flops_only_at_burst_peak_ms": round(1e3 * fl_all / peak_b, 4),
            "frac_of_flops_only": round(1e3 * fl_all / peak_b / meas, 4) if meas > 0 else None,
            "note": "at_roofline_ms sums, per stage, the slower of flops at the sustained "
                    "compute peak and the method's bytes at the HBM bandwidth"}


def traffic_from_profiles(stage, prec, workload):
    """DRAM bytes per launch of a stage's kernel from the committed ncu capture
    of that stage, precision and workload shape (profiles/traffic.json), or
    None where there is none."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        v = d.get(f"{stage}:{prec}:{workload}")
        return None if v is None else v.get("bytes_per_launch")
    except Exception:
        return None


def rank_seed(seed: int, rank: int) -> int:
    """Each rank runs its own independent stream (its own planted tensor)."""
    return seed + 1000 * rank


def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's value (no-op for one rank)."""
    if world <= 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


@contextlib.contextmanager
def no_gc():
    """The interpreter's cycle collector stays off inside a timed region (a
    collection pass can stall the host for tens of milliseconds, which would be
    charged to the library); garbage is collected before it starts."""
    gc.collect()
    gc.disable()
    try:
        yield
    finally:
        gc.enable()


def whole_job_rate(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    return world * units_per_rank / seconds_max


def run_stream(args, wl, prec, steps, warmup, rank, world, time_e2e):
    import torch

    import paper_1807_01350_gb300 as pkg

    dev = torch.device("cuda", torch.cuda.current_device())
    nbd = min(steps, 3)   # extra appends with per-stage events (the stage breakdown)
    nb = warmup + steps + nbd + (max(steps, 2) if time_e2e else 0)
    d = stream_inputs(wl, prec, rank_seed(args.seed, rank), nb, dev)
    stream = torch.cuda.current_stream()
    g = pkg.Octen(wl.I, wl.J, wl.R, wl.P, wl.Q, wl.S, wl.als_iters, prec, stream=stream)
    t_old, t = wl.t_old, wl.batch
    g.init(d["X"][:t_old], d["U"], d["V"], d["W"][0], d["A0"], d["B0"], d["C0"])
    k = t_old
    for b in range(warmup):
        g.append(d["X"][k:k + t], d["W"][1 + b])
        k += t
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = pkg.launch_count()
    tc0 = pkg.tc_launch_count()
    fb0 = pkg.tc_fallback_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk, no_gc():
        torch.cuda.synchronize()
        ev0.record(stream)
        for s in range(steps):
            g.append(d["X"][k:k + t], d["W"][1 + warmup + s])
            k += t
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = pkg.launch_count() - launches0
    tc_launches = pkg.tc_launch_count() - tc0
    tc_fallbacks = pkg.tc_fallback_count() - fb0
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    if world > 1:
        torch.distributed.barrier()
    # stage breakdown: further appends with CUDA events around every stage
    # (launched one by one, since the events sit between the kernels)
    g.reset_stage_times()
    g.set_timing(True)
    for s in range(nbd):
        g.append(d["X"][k:k + t], d["W"][1 + warmup + steps + s])
        k += t
    torch.cuda.synchronize()
    g.set_timing(False)
    stages = g.stage_times()
    fit = g.fit(d["X"][:k])
    # the two tensor-core contractions run once per append when the path is taken
    tc_stages = ("mode2", "mode1") if tc_launches >= 2 * steps else ()
    if tc_launches >= (2 + 2 * wl.als_iters + 1) * steps:
        tc_stages = tc_stages + ("als_gemm",)
    out = dict(ms=ms, steps=steps, slices=steps * t, stages=stages, stage_steps=nbd, fit=fit,
               launches=launches, tc_launches=tc_launches, tc_fallbacks=tc_fallbacks,
               tc_stages=tc_stages,
               clocks=clk.summary())
    if time_e2e:
        out["e2e"] = run_e2e(g, d, wl, prec, k, steps, warmup, rank, world)
    g.close()
    del d
    torch.cuda.empty_cache()
    return out


def read_factors(g, Ah, Bh, Ch):
    """Reads A, B and every row of C so far into the caller's host buffers.
    Ch is sized once for the stream's final row count; the rows the context
    holds now are its leading rows (a contiguous prefix, which the binding
    accepts as a C of exactly that many rows).  Returns the row count."""
    return g.factors_into(Ah, Bh, Ch[:g.rows])


def run_e2e(g, d, wl, prec, k, steps, warmup, rank, world):
    """The same appends through the public API with pinned HOST buffers, as a
    serving loop runs them: step s enqueues its batch with octen_append_async
    (the library copies it from pinned host memory in pieces and copies A, B
    and the new rows of C back into pinned host buffers when the append has
    run), then waits for step s - 2, two appends in flight.  Every step's time
    thus includes its host-to-device copy and its device-to-host read, and
    the copy of one batch overlaps the updates before it.  Each step has its
    own input and output buffers until it has been waited for (three sets in
    turn).  The synchronous form (octen_append then octen_get_factors every
    step, nothing overlapped) is timed beside it."""
    import torch

    t = wl.batch
    depth = 2
    hostX = [d["X"][k + i * t:k + (i + 1) * t].to("cpu").pin_memory() for i in range(2)]
    hostX.append(hostX[0].clone().pin_memory())
    hostW = [d["W"][1 + warmup + i].to("cpu").pin_memory() for i in range(steps)]
    K_end = k + (warmup + 2 * steps) * t
    Ah = torch.empty((wl.I, wl.R), dtype=torch.float32).pin_memory()
    Bh = torch.empty((wl.J, wl.R), dtype=torch.float32).pin_memory()
    Ch = torch.empty((K_end, wl.R), dtype=torch.float32).pin_memory()
    outs = [(torch.empty((wl.I, wl.R), dtype=torch.float32).pin_memory(),
             torch.empty((wl.J, wl.R), dtype=torch.float32).pin_memory(),
             torch.empty((t, wl.R), dtype=torch.float32).pin_memory())
            for _ in range(depth + 1)]
    xb = hostX[0].numel() * hostX[0].element_size()
    wb = hostW[0].numel() * 4
    ptrs = lambda o: [a.data_ptr() for a in o]
    # untimed warm-up appends through the same host path (the first one from
    # host buffers tunes the GEMMs of the piecewise copy's shapes)
    for s in range(warmup):
        tk = g.append_async_ptr(hostX[s % 2].data_ptr(), t, hostW[s % steps].data_ptr(),
                                *ptrs(outs[s % 2]))
        g.wait(tk)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    with no_gc():
        t0 = time.perf_counter()
        tickets = []
        for s in range(steps):
            tickets.append(g.append_async_ptr(hostX[s % 3].data_ptr(), t, hostW[s].data_ptr(),
                                              *ptrs(outs[s % 3])))
            if len(tickets) > depth:
                g.wait(tickets[-1 - depth])
        for tk in tickets[-depth:]:
            g.wait(tk)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
    sec = max_over_ranks(sec, world, torch.device("cuda"))
    d2h = (wl.I + wl.J + t) * wl.R * 4
    # the synchronous form, for comparison
    d2h_sync = 0
    with no_gc():
        t0 = time.perf_counter()
        for s in range(steps):
            g.append_ptr(hostX[s % 2].data_ptr(), t, hostW[s].data_ptr())
            kk = read_factors(g, Ah, Bh, Ch)
            d2h_sync += (wl.I + wl.J + kk) * wl.R * 4
        torch.cuda.synchronize()
        sec_sync = time.perf_counter() - t0
    sec_sync = max_over_ranks(sec_sync, world, torch.device("cuda"))
    return {"value": round(whole_job_rate(steps * t, sec, world), 3), "unit": "slices/s",
            "h2d_bytes_per_step": int(xb + wb), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": round(1e3 * sec / steps, 3),
            "api": "octen_append_async from pinned host batches, step s waiting for step s-2; "
                   "A, B and the new C rows copied back into pinned host buffers every step",
            "sync": {"value": round(whole_job_rate(steps * t, sec_sync, world), 3),
                     "ms_per_step": round(1e3 * sec_sync / steps, 3),
                     "d2h_bytes_per_step": int(d2h_sync / steps),
                     "api": "octen_append then octen_get_factors (all of C) every step"}}


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
class OracleSampler:
    """The FP64 oracle on a bounded sample of one append of the workload.

    Setup (untimed): the workload's factors, projections and a batch of new
    slices, and the oracle's state from one existing slice.  Timed pieces:
    `replica(p)` = compression of the batch into replica p + its CP-ALS +
    anchor match; `lift()` = the lift of A and B and the solve of the new rows
    of C.  One append costs P replica pieces plus one lift."""

    def __init__(self, wl, seed=0, prec=None):
        import oracle

        self.o_mod = oracle
        self.wl = wl
        self.prec = prec or wl.prec
        I, J, R, P, Q, S, t = wl.I, wl.J, wl.R, wl.P, wl.Q, wl.S, wl.batch
        A, B, C = factors(I, J, 1 + t, R, seed, cond=wl.cond, big_frac=wl.big_frac)
        # the slices as the library receives them (bf16 unless fp32)
        self.X = round_to(slice_batch(A, B, C, 0, 1 + t, wl.noise, seed),
                          "fp32" if self.prec == "fp32" else "bf16")
        U, V = projections(I, J, P, Q, S, seed, self.prec)
        Wo = time_projection(1, P, Q, S, seed, -1)
        Wn = time_projection(t, P, Q, S, seed, 0)
        A0, B0, C0 = init_factors(A, B, C[:1], 0.01, seed)
        self.inputs = dict(U=U, V=V, Wo=Wo, Wn=Wn, A0=A0, B0=B0, C0=C0)
        self.Wn = Wn
        self.o = oracle.OctenOracle(I, J, R, P, Q, S, wl.als_iters)
        self.o.init(self.X[:1], U, V, Wo, A0, B0, C0)
        self.Wp = [oracle.replica_block(Wn, p, Q, S) for p in range(P)]
        self.ref_a = (self.o.U[0].T @ self.o.A)[:S]
        self.ref_b = (self.o.V[0].T @ self.o.B)[:S]
        self.hats = {}

    def replica(self, p):
        o, O, wl = self.o, self.o_mod, self.wl
        t0 = time.perf_counter()
        Yp = o.Y[p] + O.compress(self.X[1:], o.U[p], o.V[p], self.Wp[p])
        At, Bt, Ct = O.cp_als(Yp, o.U[p].T @ o.A, o.V[p].T @ o.B, wl.als_iters)
        self.hats[p] = O.align(At, Bt, Ct, self.ref_a, self.ref_b, wl.S)
        return time.perf_counter() - t0

    def lift(self):
        o, O, P = self.o, self.o_mod, self.wl.P
        if not self.hats:
            self.replica(0)
        hats = [self.hats.get(p, next(iter(self.hats.values()))) for p in range(P)]
        t0 = time.perf_counter()
        O.lift_factor(o.A, o.U, [h[0] for h in hats])
        O.lift_factor(o.B, o.V, [h[1] for h in hats])
        O.lift_C(self.Wp, [h[2] for h in hats], o.G)
        return time.perf_counter() - t0

    def full_append(self):
        """The oracle's whole append of the batch (every replica, the lift);
        returns its wall time.  Changes the oracle's state."""
        t0 = time.perf_counter()
        self.o.append(self.X[1:], self.Wn)
        return time.perf_counter() - t0

    def gpu_parity(self, pkg, prec):
        """The library on the same inputs (init from the same slice, the same
        append): worst replica summary error, the fits and the factor-match
        score against the oracle's state after full_append()."""
        import torch

        wl, d, o, O = self.wl, self.inputs, self.o, self.o_mod
        dev = torch.device("cuda", torch.cuda.current_device())
        f32 = lambda a: torch.as_tensor(np.asarray(a, np.float32), device=dev)
        xs = f32(self.X).to(torch.float32 if prec == "fp32" else torch.bfloat16)
        g = pkg.Octen(wl.I, wl.J, wl.R, wl.P, wl.Q, wl.S, wl.als_iters, prec)
        g.init(xs[:1], f32(d["U"]), f32(d["V"]), f32(d["Wo"]), f32(d["A0"]), f32(d["B0"]),
               f32(d["C0"]))
        g.append(xs[1:], f32(d["Wn"]))
        Y = g.replicas()
        A, B, C = g.factors()
        fit_gpu = g.fit(xs)
        g.close()
        err = max(float(np.linalg.norm(Y[p] - o.Y[p]) / np.linalg.norm(o.Y[p]))
                  for p in range(wl.P))
        fit_ref = O.fit(self.X, o.A, o.B, o.C)
        return {"replica_rel_err_max": round(err, 7),
                "fit": round(fit_gpu, 6), "fit_oracle": round(fit_ref, 6),
                "fit_delta": round(fit_gpu - fit_ref, 6),
                "meets_fit_qualifier": bool(fit_gpu >= fit_ref - 1e-3),
                "fms": round(_fms((A, B, C), (o.A, o.B, o.C)), 6),
                "oracle_inputs": "fp32-rounded slices" if prec == "fp32" else "bf16 slices",
                "case": f"{wl.name} shapes, {prec}: init from 1 slice, one append of {wl.batch}"}

    def describe(self, timed_p, t_rep, t_lift):
        """What a reference-arm run timed: `timed_p` lists the replica of every
        timed piece (replica s mod P at step s)."""
        wl = self.wl
        distinct = len(set(timed_p))
        return (f"{len(timed_p)} replica pieces (compression + CP-ALS + anchor match of one "
                f"replica of a {wl.batch}-slice append at {wl.name}) over {distinct} distinct "
                f"replicas of {wl.P}, {t_rep:.2f} s per piece on average; the value extrapolates "
                f"one append as {wl.P} pieces plus the full lift of A, B and the new C rows "
                f"({t_lift:.2f} s, timed once)")


def _fms(model, ref):
    """Factor-match score: mean over matched columns of the product over modes
    of |cos|, columns matched by the assignment that maximises the sum."""
    from scipy.optimize import linear_sum_assignment

    sim = np.ones((ref[0].shape[1],) * 2)
    for F, G in zip(model, ref):
        F = np.asarray(F, np.float64)
        G = np.asarray(G, np.float64)
        nf, ng = np.linalg.norm(F, axis=0), np.linalg.norm(G, axis=0)
        sim = sim * np.abs(F.T @ G) / np.outer(np.where(nf > 0, nf, 1), np.where(ng > 0, ng, 1))
    rows, cols = linear_sum_assignment(-sim)
    return float(sim[rows, cols].mean())


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def cpu_cores():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    return os.cpu_count()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c4", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--beside", default="fp32,fp8", help="other precisions timed beside")
    ap.add_argument("--beside-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--uneven-streams", type=int, default=0,
                    help="the batched uneven-streams workload with this many streams (64 in the "
                         "configuration): one append per stream per step through octen_append_many")
    ap.add_argument("--replay", type=int, default=0,
                    help="replay a stream of this many slices through appends of the workload's "
                         "batch size (the scalability runs; e.g. --workload q3_100 --replay 1000000)")
    ap.add_argument("--profile-case", action="store_true",
                    help="one append of --slices slices on the workload's shapes with 4 existing "
                         "slices, kernels launched one by one (small case for profiler captures)")
    ap.add_argument("--compress-only", action="store_true",
                    help="time octen_compress alone on --slices slices (profiling case)")
    ap.add_argument("--nmode", default="",
                    help="the N-mode extension's workload of this name (n4_100, n5_30): appends "
                         "through the octen_n_* path, with the FP64 N-mode oracle beside it")
    ap.add_argument("--slices", type=int, default=4)
    ap.add_argument("--existing", type=int, default=0,
                    help="override the number of existing slices (small profiling cases)")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.existing > 0:
        import dataclasses
        wl = dataclasses.replace(wl, t_old=args.existing)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    args.warmup = max(args.warmup, 3)
    if args.steps < 1:
        ap.error("--steps must be at least 1")

    if args.impl == "reference":
        return main_reference(args, wl, world, rank)
    if args.nmode:
        return main_nmode(args)
    if args.uneven_streams:
        return main_uneven(args)
    if args.replay:
        return main_replay(args, wl)
    if args.profile_case:
        return main_profile_case(args, wl)
    if args.compress_only:
        return main_compress_only(args, wl)

    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1807_01350_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_1807_01350_gb300  # noqa: F401  (fails loudly without the CUDA library)

    main_run = run_stream(args, wl, args.prec, args.steps, args.warmup, rank, world,
                          time_e2e=not args.no_e2e)
    beside = {}
    for prec in [p for p in args.beside.split(",") if p and p != args.prec]:
        r = run_stream(args, wl, prec, args.beside_steps, 3, rank, world, time_e2e=False)
        beside[prec] = {"value": round(whole_job_rate(r["slices"], r["ms"] / 1e3, world), 3),
                        "ms_per_step": round(r["ms"] / r["steps"], 3), "fit": round(r["fit"], 6),
                        "steps": r["steps"],
                        "stage_ms_per_step": {k: round(v[0] / r["stage_steps"], 3)
                                              for k, v in r["stages"].items() if v[1]}}
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return

    pk = peaks()
    st = main_run["stages"]
    timed = {k: v for k, v in st.items() if v[1] > 0}
    dominant = max(("mode2", "mode1", "mode3", "als_gemm"), key=lambda s: st[s][0])
    ms_launch = st[dominant][0] / st[dominant][1]
    tcs = main_run["tc_stages"]
    roof = roofline_for(dominant, ms_launch, wl, args.prec, pk,
                        traffic_from_profiles(dominant, args.prec, wl.name), tcs)
    comp = {s: roofline_for(s, st[s][0] / st[s][1], wl, args.prec, pk,
                            traffic_from_profiles(s, args.prec, wl.name), tcs)
            for s in ("quantize", "mode2", "mode1", "mode3", "als_gemm") if st[s][1]}
    # the compression as a whole (quantise, mode 2, mode 1, mode 3)
    compression_roofline = compression_at_roofline(wl, args.prec, pk, comp, tcs)
    value = whole_job_rate(main_run["slices"], main_run["ms"] / 1e3, world)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "slices/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(main_run["ms"] / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
        "data": "synthetic planted-CP slices (seeded), resident in HBM",
        "config": {"workload": wl.name, "I": wl.I, "J": wl.J, "R": wl.R, "P": wl.P, "Q": wl.Q,
                   "S": wl.S, "batch_slices": wl.batch, "existing_slices": wl.t_old,
                   "als_iters": wl.als_iters, "noise": wl.noise,
                   "l2": "inputs larger than L2 (each batch is a fresh "
                         f"{wl.batch * wl.I * wl.J * (4 if args.prec == 'fp32' else 2) / 2**20:.0f} MiB)",
                   "parallelism": f"independent stream per GPU x{world}"},
        "fit": round(main_run["fit"], 6),
        "clocks": main_run["clocks"],
        "gpu_launches": main_run["launches"],
        "tcgen05_launches": main_run["tc_launches"],
        "tcgen05_fallbacks": main_run["tc_fallbacks"],
        "roofline": roof,
        "stage_ms_per_step": {k: round(v[0] / main_run["stage_steps"], 3)
                              for k, v in timed.items()},
        "stage_note": "per-stage CUDA events on separate appends launched one by one",
        "stage_roofline": comp,
        "compression_roofline": compression_roofline,
        "beside": beside,
    }
    if "e2e" in main_run:
        line["e2e"] = main_run["e2e"]
    if world == 1 and not args.no_cpu_baseline:
        smp = OracleSampler(wl, args.seed, args.prec)
        sec = smp.full_append()
        line["cpu_baseline"] = {
            "value": round(wl.batch / sec, 5), "unit": "slices/s", "cores": cpu_cores(), "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": f"one whole append of {wl.batch} slices at {wl.name} ({args.prec} inputs) "
                      f"after an init from 1 slice: compression and CP-ALS of all {wl.P} "
                      f"replicas, anchor match, lift ({sec:.1f} s)"}
        import paper_1807_01350_gb300 as pkg
        line["parity"] = smp.gpu_parity(pkg, args.prec)
        # every other precision's error against the FP64 oracle on its own
        # inputs (fp32 slices for fp32, the bf16 slices for bf16 and fp8)
        for prec in beside:
            sp = OracleSampler(wl, args.seed, prec)
            sp.full_append()
            beside[prec]["parity"] = sp.gpu_parity(pkg, prec)
    print(json.dumps(line), flush=True)


def main_uneven(args):
    """The batched uneven-streams workload: n independent decompositions of
    different shapes, ranks and batch sizes, each on its own CUDA stream; a step
    is one append on every stream through octen_append_many (all enqueued
    before any is waited for).  Compared with the same n updates in FP32, one
    after another (octen_append per stream)."""
    # one hardware work queue per stream (the default of 8 queues would make
    # the 64 streams share queues and wait on one another's launches); read
    # when the CUDA context is created, so set before the first CUDA call
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch

    from paper_1807_01350_gb300 import build as B
    B.build()
    import paper_1807_01350_gb300 as pkg

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cfgs = uneven_streams(args.uneven_streams, args.seed)
    f32 = lambda a: torch.as_tensor(np.asarray(a, np.float32), device=dev)
    streams = []   # one CUDA stream per decomposition, alive as long as its context

    def make(prec):
        dt = torch.float32 if prec == "fp32" else torch.bfloat16
        ctxs, batches, ws = [], [], []
        streams.clear()
        for wl, sd in cfgs:
            A, B_, C = factors(wl.I, wl.J, wl.t_old + 2 * wl.batch, wl.R, sd)
            U, V = projections(wl.I, wl.J, wl.P, wl.Q, wl.S, sd, prec)
            A0, B0, C0 = init_factors(A, B_, C[:wl.t_old], 0.01, sd)
            streams.append(torch.cuda.Stream())
            g = pkg.Octen(wl.I, wl.J, wl.R, wl.P, wl.Q, wl.S, wl.als_iters, prec,
                          stream=streams[-1])
            X0 = slice_batch_torch(A, B_, C, 0, wl.t_old, wl.noise, sd, dev, dt)
            g.init(X0, f32(U), f32(V), f32(time_projection(wl.t_old, wl.P, wl.Q, wl.S, sd, -1)),
                   f32(A0), f32(B0), f32(C0))
            del X0
            ctxs.append(g)
            batches.append([slice_batch_torch(A, B_, C, wl.t_old + b * wl.batch,
                                              wl.t_old + (b + 1) * wl.batch, wl.noise, sd, dev, dt)
                            for b in range(2)])
            ws.append([f32(time_projection(wl.batch, wl.P, wl.Q, wl.S, sd, b)) for b in range(2)])
        torch.cuda.synchronize()
        return ctxs, batches, ws

    slices = sum(wl.batch for wl, _ in cfgs)
    ctxs, batches, ws = make("bf16")
    warm, steps = max(args.warmup, 3), args.steps
    for s in range(warm):
        pkg.append_many(ctxs, [b[s % 2] for b in batches], [w[s % 2] for w in ws])
    torch.cuda.synchronize()
    with ClockSampler(0) as clk, no_gc():
        t0 = time.perf_counter()
        for s in range(steps):
            pkg.append_many(ctxs, [b[s % 2] for b in batches], [w[s % 2] for w in ws])
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
    for g in ctxs:
        g.close()
    del ctxs, batches, ws
    torch.cuda.empty_cache()
    # the FP32 comparison: the same streams, one update after another
    ctxs, batches, ws = make("fp32")
    for g, b, w in zip(ctxs, batches, ws):
        g.append(b[0], w[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g, b, w in zip(ctxs, batches, ws):
        g.append(b[1], w[1])
    torch.cuda.synchronize()
    sec32 = time.perf_counter() - t0
    for g in ctxs:
        g.close()
    value = slices * steps / sec
    print(json.dumps({
        "metric": METRIC, "value": round(value, 3), "unit": "slices/s", "n_gpus": 1,
        "steps": steps, "warmup": warm, "ms_per_step": round(1e3 * sec / steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic planted-CP slices (seeded), resident in HBM",
        "config": {"workload": f"c5_uneven_streams_x{len(cfgs)}", "streams": len(cfgs),
                   "slices_per_step": slices,
                   "shapes": [[wl.I, wl.J, wl.R, wl.batch, wl.Q] for wl, _ in cfgs[:8]],
                   "parallelism": "one CUDA stream per decomposition, octen_append_many"},
        "clocks": clk.summary(),
        "fp32_sequential": {"value": round(slices / sec32, 3), "unit": "slices/s",
                            "ms_per_step": round(1e3 * sec32, 3),
                            "note": "the same updates in fp32, octen_append one stream after another"},
        "speedup_vs_fp32_sequential": round(value / (slices / sec32), 3)}), flush=True)


def ncompress_flops(wl, t):
    """Multiply-adds x 2 of the N-mode compression chain for t slices: the first
    product over every slice for all P Q columns, the per-replica products of
    the other non-temporal modes, the time contraction."""
    dims, P, Q = list(wl.dims), wl.P, wl.Q
    rows = t * int(np.prod(dims[:-1]))
    fl = 2.0 * rows * dims[-1] * P * Q
    elems = rows * Q
    for m in range(len(dims) - 2, -1, -1):
        rin = elems // dims[m]
        fl += 2.0 * P * rin * Q * dims[m]
        elems = rin * Q
    fl += 2.0 * P * (elems // t) * Q * t
    return fl


def nals_flops(wl):
    """Algorithmic flops of the replica CP-ALS of one append: per update an
    N-way MTTKRP (2 Q^N R) and the R x R solve applied to Q rows (2 Q R^2)."""
    N, Q, R = len(wl.dims) + 1, wl.Q, wl.R
    per_update = 2.0 * Q ** N * R + 2.0 * Q * R * R
    return wl.P * (wl.als_iters * N + 1) * per_update


def main_nmode(args):
    """The N-mode extension (Sec. "Extending to Higher-Order Tensors"): a
    stream of appends of the workload's batch size through octen_n_append with
    the slices resident in HBM; the FP64 N-mode oracle runs the first append
    beside it (parity and the CPU baseline)."""
    import torch

    from paper_1807_01350_gb300 import build as B
    B.build()
    import paper_1807_01350_gb300 as pkg
    from oracle import octen_n
    from synth import NWORKLOADS, nfactors, ninit_factors, nprojections, nslice_batch

    wl = NWORKLOADS[args.nmode]
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    nb, t, t_old = 4, wl.batch, wl.t_old
    K = t_old + nb * t
    As, C = nfactors(wl.dims, K, wl.R, args.seed)
    X = round_to(nslice_batch(As, C, 0, K, wl.noise, args.seed), "fp32")
    Us = nprojections(wl.dims, wl.P, wl.Q, wl.S, args.seed)
    A0s, C0 = ninit_factors(As, C[:t_old], 0.01, args.seed)
    Ws = [time_projection(t_old, wl.P, wl.Q, wl.S, args.seed, -1)] + \
        [time_projection(t, wl.P, wl.Q, wl.S, args.seed, b) for b in range(nb)]
    f32 = lambda a: torch.as_tensor(np.asarray(a, np.float32), device=dev)
    Xd = f32(X)
    Wd = [f32(w) for w in Ws]
    batches = [Xd[t_old + b * t:t_old + (b + 1) * t] for b in range(nb)]

    def fresh():
        g = pkg.OctenN(wl.dims, wl.R, wl.P, wl.Q, wl.S, wl.als_iters)
        g.init(Xd[:t_old], [f32(u) for u in Us], Wd[0], [f32(a) for a in A0s], f32(C0))
        return g

    # parity of the first append against the oracle
    g = fresh()
    g.append(batches[0], Wd[1])
    A_gpu, C_gpu = g.factors()
    g.close()
    o = octen_n.OctenOracleN(list(wl.dims), wl.R, wl.P, wl.Q, wl.S, wl.als_iters)
    o.init(X[:t_old], Us, Ws[0], A0s, C0)
    t0 = time.perf_counter()
    o.append(X[t_old:t_old + t], Ws[1])
    cpu_sec = time.perf_counter() - t0
    relf = lambda x, y: float(np.linalg.norm(x - y) / np.linalg.norm(y))
    f_gpu = octen_n.fit_n(X[:t_old + t], A_gpu, C_gpu)
    f_ref = octen_n.fit_n(X[:t_old + t], o.A, o.C)
    parity = {"A_rel_err_max": max(relf(a, b) for a, b in zip(A_gpu, o.A)),
              "C_rel_err": relf(C_gpu, o.C), "fit_gpu": round(f_gpu, 6),
              "fit_oracle": round(f_ref, 6), "tol": {"F": 1e-3, "fit": 1e-4},
              "ok": bool(max(relf(a, b) for a, b in zip(A_gpu, o.A)) < 1e-3 and
                         relf(C_gpu, o.C) < 1e-3 and abs(f_gpu - f_ref) < 1e-4)}

    # timed stream
    g = fresh()
    warm, steps = max(args.warmup, 3), args.steps
    for s in range(warm):
        g.append(batches[s % nb], Wd[1 + s % nb])
    torch.cuda.synchronize()
    l0 = pkg.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk, no_gc():
        e0.record()
        for s in range(steps):
            g.append(batches[s % nb], Wd[1 + s % nb])
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = pkg.launch_count() - l0
    # stage breakdown on further appends with the stage timers on
    g.set_timing(True)
    for s in range(nb):
        g.append(batches[s % nb], Wd[1 + s % nb])
    st = g.stage_times()
    g.close()
    pk = peaks()
    stage_ms = {k: v[0] / v[1] for k, v in st.items() if v[1]}
    work = {"compress": ncompress_flops(wl, t), "als": nals_flops(wl)}
    stage_roof = {}
    for k, fl in work.items():
        a = fl / (stage_ms[k] / 1e3) / 1e12
        stage_roof[k] = {"bound": "alu", "achieved": round(a, 3), "peak": round(FP32_ALU_TFLOPS, 1),
                         "unit": "TFLOP/s", "frac": round(a / FP32_ALU_TFLOPS, 4),
                         "flops_per_launch": fl, "ms_per_launch": round(stage_ms[k], 4),
                         "traffic": None}
    dominant = max(work, key=lambda k: stage_ms[k])
    value = steps * t / (ms / 1e3)
    print(json.dumps({
        "metric": "new slices/sec, N-mode online CP update (fp32)", "value": round(value, 3),
        "unit": "slices/s", "n_gpus": 1, "steps": steps, "warmup": warm,
        "ms_per_step": round(ms / steps, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic planted N-mode CP slices (seeded), resident in HBM",
        "config": {"workload": wl.name, "N": len(wl.dims) + 1, "dims": list(wl.dims),
                   "R": wl.R, "P": wl.P, "Q": wl.Q, "S": wl.S, "batch_slices": t,
                   "existing_slices": t_old, "als_iters": wl.als_iters,
                   "l2": f"{nb} batches of {t * wl.slice_elems * 4 / 2**20:.0f} MiB cycled"},
        "clocks": clk.summary(), "gpu_launches": launches,
        "roofline": dict(stage_roof[dominant], kernel=dominant),
        "stage_ms_per_step": {k: round(v, 4) for k, v in stage_ms.items()},
        "stage_roofline": stage_roof,
        "cpu_baseline": {"value": round(t / cpu_sec, 5), "unit": "slices/s", "cores": cpu_cores(), "cpu_model": cpu_model(),
                         "kind": "oracle",
                         "sample": f"one whole append of {t} slices at {wl.name} after an init "
                                   f"from {t_old} slices ({cpu_sec:.1f} s)"},
        "parity": parity}), flush=True)


def main_replay(args, wl):
    """Algorithm 1 over a long stream (the scalability replay of Sec. "[Q3]
    Scalability Evaluation"): init from the workload's existing slices, then
    appends of its batch size until --replay slices in all.  Slices are drawn on
    the GPU a window at a time (outside the timed appends); each window's
    appends are timed with CUDA events, so the time per append along the stream
    shows how the cost grows with K."""
    import torch

    from paper_1807_01350_gb300 import build as B
    B.build()
    import paper_1807_01350_gb300 as pkg

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    K, t, t_old = args.replay, wl.batch, wl.t_old
    A, B_, C = factors(wl.I, wl.J, K, wl.R, args.seed, cond=wl.cond, big_frac=wl.big_frac)
    U, V = projections(wl.I, wl.J, wl.P, wl.Q, wl.S, args.seed, args.prec)
    W0 = time_projection(t_old, wl.P, wl.Q, wl.S, args.seed, -1)
    A0, B0, C0 = init_factors(A, B_, C[:t_old], 0.01, args.seed)
    dt = torch.float32 if args.prec == "fp32" else torch.bfloat16
    f32 = lambda a: torch.as_tensor(np.asarray(a, np.float32), device=dev)
    g = pkg.Octen(wl.I, wl.J, wl.R, wl.P, wl.Q, wl.S, wl.als_iters, args.prec)
    g.init(slice_batch_torch(A, B_, C, 0, t_old, wl.noise, args.seed, dev, dt), f32(U), f32(V),
           f32(W0), f32(A0), f32(B0), f32(C0))
    window = 1000   # appends per timed window
    k, b, total_ms, windows = t_old, 0, 0.0, []
    with ClockSampler(0) as clk, no_gc():
        while k + t <= K:
            n = min(window, (K - k) // t)
            X = slice_batch_torch(A, B_, C, k, k + n * t, wl.noise, args.seed, dev, dt)
            Ws = [f32(time_projection(t, wl.P, wl.Q, wl.S, args.seed, b + i)) for i in range(n)]
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for i in range(n):
                g.append(X[i * t:(i + 1) * t], Ws[i])
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            total_ms += ms
            k += n * t
            b += n
            windows.append([k, round(ms / n, 4)])
            del X, Ws
    g.close()
    slices = k - t_old
    print(json.dumps({
        "metric": METRIC, "value": round(slices / (total_ms / 1e3), 3), "unit": "slices/s",
        "n_gpus": 1, "steps": b, "ms_per_step": round(total_ms / b, 4),
        "higher_is_better": True, "dtype": args.prec, "data": "synthetic planted-CP slices (seeded)",
        "config": {"workload": wl.name, "I": wl.I, "J": wl.J, "R": wl.R, "P": wl.P, "Q": wl.Q,
                   "S": wl.S, "batch_slices": t, "existing_slices": t_old, "K": k,
                   "als_iters": wl.als_iters},
        "clocks": clk.summary(),
        "replay": {"note": "time per append (ms) after each window of appends, by slices so far",
                   "ms_per_append_by_K": windows}}), flush=True)


def main_profile_case(args, wl):
    """Init from 4 existing slices and one append of --slices new slices on the
    workload's shapes (every kernel of an append at full size, a few GB on the
    device), with the CP-ALS launched kernel by kernel rather than as a graph."""
    os.environ["OCTEN_GRAPH"] = "0"
    import torch

    from paper_1807_01350_gb300 import build as B
    B.build()
    import paper_1807_01350_gb300 as pkg

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    t_old, t = 4, args.slices
    A, B_, C = factors(wl.I, wl.J, t_old + t, wl.R, args.seed, cond=wl.cond,
                       big_frac=wl.big_frac)
    U, V = projections(wl.I, wl.J, wl.P, wl.Q, wl.S, args.seed, args.prec)
    W0 = time_projection(t_old, wl.P, wl.Q, wl.S, args.seed, -1)
    W1 = time_projection(t, wl.P, wl.Q, wl.S, args.seed, 0)
    A0, B0, C0 = init_factors(A, B_, C[:t_old], 0.01, args.seed)
    dt = torch.float32 if args.prec == "fp32" else torch.bfloat16
    X = slice_batch_torch(A, B_, C, 0, t_old + t, wl.noise, args.seed, dev, dt)
    f32 = lambda a: torch.as_tensor(np.asarray(a, np.float32), device=dev)
    g = pkg.Octen(wl.I, wl.J, wl.R, wl.P, wl.Q, wl.S, wl.als_iters, args.prec)
    g.init(X[:t_old], f32(U), f32(V), f32(W0), f32(A0), f32(B0), f32(C0))
    n0 = pkg.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.append(X[t_old:], f32(W1))
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"mode": "profile_case", "workload": wl.name, "prec": args.prec,
                      "slices": t, "append_ms": round(e0.elapsed_time(e1), 3),
                      "launches": pkg.launch_count() - n0}), flush=True)
    g.close()


def main_compress_only(args, wl):
    """Stateless compression of a few slices of the workload (a small, fixed
    case for profiler captures): prints one JSON line with the time per call."""
    import torch

    from paper_1807_01350_gb300 import build as B
    B.build()
    import paper_1807_01350_gb300 as pkg

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    t = args.slices
    A, B_, C = factors(wl.I, wl.J, t, wl.R, args.seed)
    U, V = projections(wl.I, wl.J, wl.P, wl.Q, wl.S, args.seed, args.prec)
    W = time_projection(t, wl.P, wl.Q, wl.S, args.seed, 0)
    dt = torch.float32 if args.prec == "fp32" else torch.bfloat16
    X = slice_batch_torch(A, B_, C, 0, t, wl.noise, args.seed, dev, dt)
    f32 = lambda a: torch.as_tensor(np.asarray(a, np.float32), device=dev)
    Ud, Vd, Wd = f32(U), f32(V), f32(W)
    ms = []
    for s in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pkg.compress(wl.I, wl.J, wl.P, wl.Q, wl.S, X, Ud, Vd, Wd, prec=args.prec)
        e1.record()
        torch.cuda.synchronize()
        if s >= args.warmup:
            ms.append(e0.elapsed_time(e1))
    print(json.dumps({"mode": "compress_only", "workload": wl.name, "prec": args.prec,
                      "slices": t, "ms_per_call": round(sum(ms) / len(ms), 3),
                      "tcgen05_launches": pkg.tc_launch_count()}), flush=True)


def main_reference(args, wl, world, rank):
    """The FP64 oracle timed on the host cores.  A step is one replica piece
    of an append (compression + CP-ALS + anchor match of one replica, replica
    s mod P at step s); ms_per_step is the mean time of a timed piece.  The
    lift, shared by all replicas, is timed once during warm-up.  The value
    extrapolates one append from those: the batch's slices over P pieces plus
    one lift."""
    if rank != 0:
        return
    smp = OracleSampler(wl, args.seed, args.prec)
    t_lift = None
    reps, timed_p = [], []
    for s in range(args.warmup + args.steps):
        p = s % wl.P
        if s < args.warmup:
            smp.replica(p)
            if t_lift is None:
                t_lift = smp.lift()
        else:
            reps.append(smp.replica(p))
            timed_p.append(p)
    t_rep = sum(reps) / len(reps)
    sec = wl.P * t_rep + t_lift
    value = wl.batch / sec
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "slices/s",
            "n_gpus": world, "steps": len(reps), "warmup": args.warmup,
            "ms_per_step": round(1e3 * t_rep, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic planted-CP slices (seeded)",
            "config": {"workload": wl.name, "I": wl.I, "J": wl.J, "R": wl.R, "P": wl.P,
                       "Q": wl.Q, "S": wl.S, "batch_slices": wl.batch,
                       "als_iters": wl.als_iters},
            "step_unit": "one replica piece of an append (compression + CP-ALS + anchor match "
                         "of one replica)",
            "extrapolated_append_ms": round(1e3 * sec, 3),
            "cpu_baseline": {"value": round(value, 5), "unit": "slices/s", "cores": cpu_cores(),
                             "cpu_model": cpu_model(), "kind": "oracle",
                             "sample": smp.describe(timed_p, t_rep, t_lift)},
            "e2e": {"value": round(value, 5), "unit": "slices/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
