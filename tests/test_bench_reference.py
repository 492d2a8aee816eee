"""The reference arm of the benchmark (the FP64 oracle on the host cores)
runs without a GPU and prints the contract's JSON line; under a multi-rank
launch only rank 0 runs it, the other ranks exit 0 without work."""
import json
import os
import subprocess
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
       "--steps", "2", "--warmup", "3"]


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    t0 = time.perf_counter()
    r = subprocess.run(CMD, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    r.wall = time.perf_counter() - t0
    return r


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "slices/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] >= 3
    assert d["config"]["workload"].startswith("c1_")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"]
    # a step is one replica piece: the timed steps fit inside the run itself,
    # and the sample says how many distinct replicas they covered
    assert d["ms_per_step"] * d["steps"] / 1e3 <= r.wall
    assert "2 distinct replicas" in cb["sample"]
    P, t = d["config"]["P"], d["config"]["batch_slices"]
    assert d["extrapolated_append_ms"] > P * d["ms_per_step"]
    assert d["value"] == pytest.approx(t / (d["extrapolated_append_ms"] / 1e3), rel=1e-3)
    assert d["e2e"] == {"value": d["value"], "unit": "slices/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]
