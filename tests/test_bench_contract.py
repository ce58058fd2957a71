"""The benchmark's reference arm (the FP64 oracle on the host cores) prints
one JSON line with every key the benchmark contract names, for the headline
workload and for the batch and weighted-BP workloads.  CPU only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def reference_line(*extra):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-seconds", "0.5", *extra], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def check_contract(d):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["data"] == "synthetic" and d["dtype"] == "f64" and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_headline_workload(oracle_mod):
    d = reference_line()
    check_contract(d)
    assert d["config"]["workload"] == "qc_n1e6_r0.02" and d["unit"] == "Mbit/s"
    # the per-core figure beside the all-core rate
    assert d["cpu_baseline"]["single_thread_s_per_frame_iter"] > 0 and d["cpu_baseline"]["single_thread_sample"]


@pytest.mark.parametrize("extra", [("--workload", "3", "--frames", "6"), ("--workload", "4")])
def test_reference_arm_other_workloads(oracle_mod, extra):
    check_contract(reference_line(*extra))
