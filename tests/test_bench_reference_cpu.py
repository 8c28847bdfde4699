"""The benchmark's reference arm on CPU: `bench.py --impl reference` times the
FP64 oracle on the host cores and prints one JSON line with the contract's keys
(the oracle is the reference: the paper ships no code).  A small workload keeps
it quick; nothing here needs a GPU."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--workload", "sinusoid64"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "sinusoid64"


def test_keep_busy_runs_steps_for_the_requested_time():
    """The untimed load before the timed region (so that the clock samples see
    the GPU under load) runs whole batches of flush + step and synchronises."""
    import time

    sys.path.insert(0, ROOT)
    import bench

    calls = {"flush": 0, "step": 0, "sync": 0}

    class Flush:
        def zero_(self):
            calls["flush"] += 1

    def step():
        calls["step"] += 1

    def sync():
        calls["sync"] += 1

    t = time.perf_counter()
    n = bench.keep_busy(step, Flush(), 0.05, sync, batch=4)
    assert time.perf_counter() - t >= 0.05
    assert n == calls["step"] == calls["flush"] and n % 4 == 0 and n >= 4
    assert calls["sync"] == n // 4
