"""bench.py's host-side legs, without a GPU: the reference arm (the oracle on
the host cores) prints the JSON line the contract asks for, the CPU baseline
takes a bounded sample, and the committed profile summaries match the kernel
sources they were taken from (else bench.py reports their traffic as null)."""
import glob
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "planetary9", "--steps", "20", "--warmup", "2"],
                         check=True, capture_output=True, text=True, cwd=ROOT).stdout
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["unit"] == bench.UNIT and line["steps"] == 20
    assert line["higher_is_better"] is True and line["config"]["n"] == 9
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_cpu_baseline_repeats_a_short_workload():
    from paper_1402_3325_gb300 import ics
    s = ics.planetary(0)
    cb = bench._cpu_baseline(s, s.dt, budget_s=2.0, max_steps=5, min_s=0.3)
    assert cb["value"] > 0 and cb["kind"] == "oracle"
    assert "passes of 5 consecutive steps" in cb["sample"]


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))),
                         ids=lambda p: os.path.basename(p))
def test_profile_summaries_match_the_current_kernel_sources(path):
    vals = {}
    with open(path) as fh:
        for ln in fh:
            if ":" in ln and ln.lstrip().startswith("- "):
                k, v = ln.lstrip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if "kernel_sources_sha256_16" not in vals:
        pytest.skip("summary without a source hash")
    name = os.path.basename(path)[:-3]
    kernel = next(k for k in ("small", "batched", "pair_step_sym_df64", "pair_step_fp64",
                              "pair_step_grp_mixed", "pair_step_grp_df64", "pair_step_grp",
                              "pair_step_sym")
                  if name.startswith(k + "_"))
    assert vals["kernel_sources_sha256_16"] == bench._kernel_sources_hash(kernel), (
        f"{name}: the kernel changed since this summary was taken")


def test_reference_arm_samples_rows_of_large_workloads(monkeypatch, capsys):
    # workloads larger than REFERENCE_ROWS particles time that many rows of
    # each step (oracle.step_sample) and count their ordered pairs
    import argparse
    monkeypatch.setattr(bench, "REFERENCE_ROWS", 64)
    args = argparse.Namespace(workload="plummer1024", steps=3, warmup=1, gpus=1)
    assert bench.run_reference(args, 0) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["config"]["n"] == 1024
    assert "64 of the 1024 rows" in line["cpu_baseline"]["sample"]
    assert line["value"] == pytest.approx(64 * 1024 * 3 / (line["ms_per_step"] * 3e-3))
