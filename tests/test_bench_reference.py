"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the
JSON contract: one line with impl "reference", the metric of the GPU arm, a
cpu_baseline describing the run, zero-byte e2e copies, and the plain dense
FP64 matvec timings.  CPU only: the arm never touches the GPU."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))


def _run(*extra):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0", *extra],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_reference_arm_times_the_plain_method_in_full():
    d = _run("--workload", "cube12_grey")
    assert d["impl"] == "reference" and d["metric"] and d["unit"] == "solves/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["N"] == 1728 and d["config"]["tol"] == 1e-10
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "no extrapolation" in cb["sample"]
    assert d["oracle_seconds_per_workload"]["extrapolated"] is False
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    mv = d["dense_matvec_fp64"]
    assert mv["12^3"]["N"] == 1728 and mv["12^3"]["ms"] > 0
    assert mv["24^3"]["N"] == 13824 and ("ms" in mv["24^3"] or "skipped" in mv["24^3"])


def test_reference_arm_extrapolates_batches_from_sampled_instances():
    d = _run("--workload", "batch8")
    assert d["config"]["instances"] == 8 and d["value"] > 0
    assert "4 of 8 instances" in d["cpu_baseline"]["sample"]
    # ms_per_step is the measured sample time, the extrapolated solve time has its own field
    assert d["oracle_seconds_per_workload"]["extrapolated"] is True
    assert d["ms_per_step"] < 600e3
