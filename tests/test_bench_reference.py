"""The benchmark's reference arm (the CPU oracle, timed on this host) prints one JSON line
with the keys the benchmark contract asks for, on every workload; the single-kernel HBM
stress workloads answer with an `unavailable` line. Runs on the CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    import time

    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    d["_wall_s"] = time.perf_counter() - t0
    return d


@pytest.mark.parametrize("workload", ["burgers1d", "advdiff1d", "batched1d", "spmv_csr", "burgers2d"])
def test_reference_line_follows_the_contract(workload):
    d = _run("--workload", workload, "--steps", "1", "--warmup", "0")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # the timed steps fit inside the run: ms_per_step is a measured (sampled) step, and the
    # scaling to the full workload is stated in the sample
    assert d["steps"] * d["ms_per_step"] / 1e3 <= d["_wall_s"]
    assert "scaled sample" in cb["sample"]


@pytest.mark.parametrize("workload", ["advdiff1d_lanes", "advdiff2d_lanes"])
def test_stress_workloads_have_no_reference(workload):
    d = _run("--workload", workload, "--steps", "1", "--warmup", "0")
    assert d["impl"] == "reference" and d["unavailable"]
